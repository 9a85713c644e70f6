"""Independent definitions of H_eff psi used to pin the sector form.

Oracle module (test infrastructure only).

1. ``apply_heff_mresolved``: expand every reduced operator into its m
   components with Clebsch-Gordan coefficients (Wigner-Eckart, CG form),
   expand the reduced psi into the uncoupled (U(1), m-resolved) product basis
   L x s1 x s2 x R, apply
       sum_i alpha_i sum_q <k q; k -q|0 0> [A x B]^k_q [C x D]^k_{-q}
   with [X x Y]^k_q = sum <kX qX; kY qY|k q> X_qX Y_qY and Jordan-Wigner
   signs in the order L, s1, s2, R, then project back on the coupled basis.
   No 6j/9j is used: this checks the C~ factors of Eq. a and the whole
   sector-task construction.
2. ``heisenberg_full_projection``: for spin chains, the block bases are built
   as explicit vectors of the 2^n-dimensional block Hilbert space from the
   same seeded MPS; H_eff = P^T H P is formed with the plain Heisenberg
   Hamiltonian and applied to psi.  This pins the renormalised block
   operators as well.
3. ``abinitio_full_projection``: the same for the ab initio Hamiltonian:
   the multiplets of both blocks and the two-site basis written out with
   Clebsch-Gordan couplings as vectors of the determinant space (one bit
   per spin-orbital, creators in ascending order, so that block x site
   products need no sign), H the full-CI matrix of the N-electron, S_z = S
   space; P^T H P pins the normal/complementary operators on truncated
   bonds too.
"""
from __future__ import annotations

import numpy as np

import synth
from . import env as envmod
from .model import IDENTITY
from .sectors import block_view
from .su2 import cg


def _mbasis(sectors):
    """m-resolved index: list of (sector, row, twoM) and a lookup."""
    idx = []
    for q, (_, S, d) in enumerate(sectors):
        for r in range(d):
            for m in range(-S, S + 1, 2):
                idx.append((q, r, m))
    return idx, {t: i for i, t in enumerate(idx)}


def _site_mbasis(site_kind):
    idx = []
    for s, (_, S) in enumerate(synth.site_states(site_kind)):
        for m in range(-S, S + 1, 2):
            idx.append((s, 0, m))
    return idx, {t: i for i, t in enumerate(idx)}


def _expand_op(blocks_or_identity, k, sectors, basis, q, is_identity=False):
    """Full matrix of component q (twos) of a reduced operator."""
    idx, look = basis
    M = np.zeros((len(idx), len(idx)))
    for i_in, (qi, ri, mi) in enumerate(idx):
        Si = sectors[qi][1]
        for i_out, (qo, ro, mo) in enumerate(idx):
            if mo != mi + q:
                continue
            So = sectors[qo][1]
            if is_identity:
                val = 1.0 if (qo == qi and ro == ri) else 0.0
            else:
                blk = blocks_or_identity.get((qo, qi))
                if blk is None:
                    continue
                val = blk[ro, ri]
            if val == 0.0:
                continue
            M[i_out, i_in] = cg(Si, mi, k, q, So, mo) * val
    return M


def _site_sectors(site_kind):
    return [(n, S, 1) for (n, S) in synth.site_states(site_kind)]


def _site_blocks(op):
    m = op.mat()
    return {(o, i): np.array([[m[o, i]]]) for o in range(m.shape[0])
            for i in range(m.shape[1]) if m[o, i] != 0.0}


def _coupled_vectors(blocks, left, right, site_kind, twoS, Lb, Sb, Rb):
    """Full-space vector of each coupled basis state with M = S.

    Returns list over psi blocks of arrays [d_a, d_b, dimL, dim1, dim2, dimR]
    would be too large; instead returns for each block a dense tensor of the
    m-structure: coefficient c[(ml), (m1), (m2), (mr)] for fixed (row, col).
    """
    sites = synth.site_states(site_kind)
    out = []
    for B in blocks:
        Sa, t1, t2, Sbb = left[B.a][1], sites[B.s1][1], sites[B.s2][1], right[B.b][1]
        coeffs = []
        for ml in range(-Sa, Sa + 1, 2):
            for m1 in range(-t1, t1 + 1, 2):
                mL1 = ml + m1
                if abs(mL1) > B.jL1:
                    continue
                c1 = cg(Sa, ml, t1, m1, B.jL1, mL1)
                if c1 == 0.0:
                    continue
                for m2 in range(-t2, t2 + 1, 2):
                    for mr in range(-Sbb, Sbb + 1, 2):
                        m2R = m2 + mr
                        if abs(m2R) > B.j2R or mL1 + m2R != twoS:
                            continue
                        c2 = cg(t2, m2, Sbb, mr, B.j2R, m2R)
                        c3 = cg(B.jL1, mL1, B.j2R, m2R, twoS, twoS)
                        c = c1 * c2 * c3
                        if c != 0.0:
                            coeffs.append((ml, m1, m2, mr, c))
        out.append(coeffs)
    return out


def apply_heff_mresolved(table, env, blocks, left, right, twoS, psi):
    sk = table.site_kind
    sites = synth.site_states(sk)
    Lb, Sb_, Rb = _mbasis(left), _site_mbasis(sk), _mbasis(right)
    nL, nS, nR = len(Lb[0]), len(Sb_[0]), len(Rb[0])
    coup = _coupled_vectors(blocks, left, right, sk, twoS, Lb, Sb_, Rb)
    # expand psi
    X = np.zeros((nL, nS, nS, nR))
    for B, coeffs in zip(blocks, coup):
        P = block_view(psi, B)
        for (ml, m1, m2, mr, c) in coeffs:
            for r in range(B.rows):
                il = Lb[1][(B.a, r, ml)]
                for cc in range(B.cols):
                    X[il, Sb_[1][(B.s1, 0, m1)], Sb_[1][(B.s2, 0, m2)], Rb[1][(B.b, cc, mr)]] += c * P[r, cc]
    # parities of the ket states along each axis
    pL = np.array([left[q][0] % 2 for (q, _, _) in Lb[0]])
    pS = np.array([sites[s][0] % 2 for (s, _, _) in Sb_[0]])
    ss = _site_sectors(sk)
    Y = np.zeros_like(X)
    for term in table.terms:
        Aop, Dop = table.left_ops[term.A], table.right_ops[term.D]
        sign = np.ones(X.shape)
        if term.B.parity:
            sign *= ((-1.0) ** pL)[:, None, None, None]
        if term.C.parity:
            sign *= ((-1.0) ** (pL[:, None] + pS[None, :]))[:, :, None, None]
        if Dop.parity:
            sign *= ((-1.0) ** (pL[:, None, None] + pS[None, :, None] + pS[None, None, :]))[:, :, :, None]
        Xs = X * sign
        k = term.k
        for q in range(-k, k + 1, 2):
            c0 = cg(k, q, k, -q, 0, 0)
            for qA in range(-Aop.k, Aop.k + 1, 2):
                qB = q - qA
                if abs(qB) > term.B.k:
                    continue
                c1 = cg(Aop.k, qA, term.B.k, qB, k, q)
                if c1 == 0.0:
                    continue
                MA = _expand_op(env.get(("L", term.A)), Aop.k, left, Lb, qA, Aop.kind == IDENTITY)
                MB = _expand_op(_site_blocks(term.B), term.B.k, ss, Sb_, qB)
                for qC in range(-term.C.k, term.C.k + 1, 2):
                    qD = -q - qC
                    if abs(qD) > Dop.k:
                        continue
                    c2 = cg(term.C.k, qC, Dop.k, qD, k, -q)
                    if c2 == 0.0:
                        continue
                    MC = _expand_op(_site_blocks(term.C), term.C.k, ss, Sb_, qC)
                    MD = _expand_op(env.get(("R", term.D)), Dop.k, right, Rb, qD, Dop.kind == IDENTITY)
                    Z = np.einsum("ai,bj,ck,dl,ijkl->abcd", MA, MB, MC, MD, Xs, optimize=True)
                    Y += term.alpha * c0 * c1 * c2 * Z
    # project back
    F = np.zeros_like(psi)
    for B, coeffs in zip(blocks, coup):
        Fb = block_view(F, B)
        for (ml, m1, m2, mr, c) in coeffs:
            for r in range(B.rows):
                il = Lb[1][(B.a, r, ml)]
                for cc in range(B.cols):
                    Fb[r, cc] += c * Y[il, Sb_[1][(B.s1, 0, m1)], Sb_[1][(B.s2, 0, m2)], Rb[1][(B.b, cc, mr)]]
    return F


# ---------------------------------------------------------------------------
# explicit full-space projection for spin-1/2 chains

def _spin_ops():
    sz = np.array([[0.5, 0.0], [0.0, -0.5]])
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])       # basis (up, down)
    return sz, sp, sp.T


def _block_states(cfg, n_sites, mps_side):
    """Explicit full-space vectors of the block multiplets with M = S... all M.

    Returns dict (sector, row, twoM) -> vector of length 2^n_sites, with the
    site order of the block as in the chain (left block: site 1 is the most
    significant factor; right block likewise left to right).
    """
    sk = synth.SPIN_HALF
    chain = synth.bond_sector_chain(cfg, n_sites)
    left = mps_side == envmod.SIDE_MPS_L
    states = {(0, 0, 0): np.array([1.0])}
    up = np.array([1.0, 0.0]); dn = np.array([0.0, 1.0])
    site_vec = {1: up, -1: dn}
    for k in range(1, n_sites + 1):
        prev, cur = chain[k - 1], chain[k]
        A = envmod.mps_tensor(cfg.seed, mps_side, k, prev, cur, sk)
        new = {}
        for qo, (rows, Q) in A.items():
            So = cur[qo][1]
            for M in range(-So, So + 1, 2):
                # coupled states |(prev row, site) So M>, stacked like Q's rows
                vecs = []
                for (qp, s, r0, dp) in rows:
                    Sp = prev[qp][1]
                    for r in range(dp):
                        v = 0.0
                        for mp in range(-Sp, Sp + 1, 2):
                            ms = M - mp
                            if abs(ms) != 1:
                                continue
                            if left:
                                c = cg(Sp, mp, 1, ms, So, M)
                                term = np.kron(states[(qp, r, mp)], site_vec[ms])
                            else:
                                c = cg(1, ms, Sp, mp, So, M)
                                term = np.kron(site_vec[ms], states[(qp, r, mp)])
                            if c != 0.0:
                                v = v + c * term
                        vecs.append(v if not np.isscalar(v) else np.zeros(2 ** k))
                V = np.array(vecs).T              # 2^k x rows
                W = V @ Q                          # 2^k x d
                for r in range(Q.shape[1]):
                    new[(qo, r, M)] = W[:, r]
        states = new
    return chain[n_sites], states


def heisenberg_full_projection(cfg, blocks, left, right, psi, J=1.0):
    """P^T H P psi for the open Heisenberg chain of cfg.L sites (small L)."""
    L = cfg.L
    nl, nr = cfg.n_left, cfg.n_right
    lsec, lst = _block_states(cfg, nl, envmod.SIDE_MPS_L)
    rsec, rst = _block_states(cfg, nr, envmod.SIDE_MPS_R)
    assert lsec == left and rsec == right
    sz, sp, sm = _spin_ops()
    dim = 2 ** L
    # full Hamiltonian as a sparse action on vectors
    def H_apply(v):
        w = np.zeros(dim)
        T = v.reshape([2] * L)
        for i in range(L - 1):
            for (Oa, Ob, c) in ((sz, sz, 1.0), (sp, sm, 0.5), (sm, sp, 0.5)):
                Z = np.tensordot(Oa, T, axes=([1], [i]))
                Z = np.moveaxis(Z, 0, i)
                Z = np.tensordot(Ob, Z, axes=([1], [i + 1]))
                Z = np.moveaxis(Z, 0, i + 1)
                w += J * c * Z.reshape(-1)
        return w
    up = np.array([1.0, 0.0]); dn = np.array([0.0, 1.0])
    site_vec = {1: up, -1: dn}
    coup = _coupled_vectors(blocks, left, right, synth.SPIN_HALF, cfg.twoS, None, None, None)
    # basis vectors of the two-site space (M = S), one per (block, row, col)
    basis = []
    for B, coeffs in zip(blocks, coup):
        for cc in range(B.cols):
            for r in range(B.rows):
                v = np.zeros(dim)
                for (ml, m1, m2, mr, c) in coeffs:
                    v += c * np.kron(np.kron(np.kron(lst[(B.a, r, ml)], site_vec[m1]), site_vec[m2]),
                                     rst[(B.b, cc, mr)])
                basis.append(v)
    P = np.array(basis).T                      # dim x psi_len, column-major block order
    return P.T @ H_apply(P @ psi), P


# ---------------------------------------------------------------------------
# ab initio: explicit block bases in the determinant space of the orbitals

# the site multiplets of a spatial orbital as vectors over its four
# occupation patterns (bit 0: spin-up, bit 1: spin-down; the doubly occupied
# pattern is c+_up c+_dn |0>), keyed by (site state, twoM)
_ORB_SITE = {(0, 0): np.eye(4)[0], (1, 1): np.eye(4)[1], (1, -1): np.eye(4)[2], (2, 0): np.eye(4)[3]}


def _orbital_block_states(seed, chain, n_orb, mps_side):
    """Explicit vectors of the multiplets (all M) of a block of n_orb orbitals
    grown by the seeded MPS over ``chain``: dict (sector, row, twoM) ->
    vector over the block's 4^n_orb occupation patterns, pattern bit
    2 j + s for local orbital j (left block: local = global orbital; right
    block: local 0 is its leftmost orbital).  Every factor is a product of
    creators in ascending spin-orbital order, so the product of a block
    state and a site state on a higher orbital is the determinant of the
    union of their patterns, with no sign."""
    sk = synth.SPATIAL_ORBITAL
    sites = synth.site_states(sk)
    left = mps_side == envmod.SIDE_MPS_L
    states = {(0, 0, 0): np.array([1.0])}
    for k in range(1, n_orb + 1):
        prev, cur = chain[k - 1], chain[k]
        A = envmod.mps_tensor(seed, mps_side, k, prev, cur, sk)
        new = {}
        for qo, (rows, Q) in A.items():
            So = cur[qo][1]
            for M in range(-So, So + 1, 2):
                vecs = []
                for (qp, s, r0, dp) in rows:
                    Sp, ts = prev[qp][1], sites[s][1]
                    for r in range(dp):
                        v = np.zeros(4 ** k)
                        for mp in range(-Sp, Sp + 1, 2):
                            ms = M - mp
                            if abs(ms) > ts:
                                continue
                            if left:     # [block x site]: the site is the highest orbital
                                c = cg(Sp, mp, ts, ms, So, M)
                                term = np.kron(_ORB_SITE[(s, ms)], states[(qp, r, mp)])
                            else:        # [site x block]: the site is the lowest orbital
                                c = cg(ts, ms, Sp, mp, So, M)
                                term = np.kron(states[(qp, r, mp)], _ORB_SITE[(s, ms)])
                            if c != 0.0:
                                v += c * term
                        vecs.append(v)
                W = np.array(vecs).T @ Q
                for r in range(Q.shape[1]):
                    new[(qo, r, M)] = W[:, r]
        states = new
    return chain[n_orb], states


def abinitio_full_projection(cfg, blocks, n, h, eri):
    """H_eff = P^T H P of the ab initio Hamiltonian (Eq. 1) for the seeded
    MPS of cfg at its middle bond, with P the explicit two-site basis
    (((L s1) j_L1 (s2 R) j_2R) S, M = S) in the N-electron, S_z = S
    determinant space, and H the full-CI matrix of that space.  Small L."""
    from . import fci
    L, N, twoS = cfg.L, cfg.N, cfg.twoS
    nl, nr = cfg.n_left, cfg.n_right
    lsec, Ls = _orbital_block_states(cfg.seed, synth.bond_sector_chain(cfg, nl), nl, envmod.SIDE_MPS_L)
    rsec, Rs = _orbital_block_states(cfg.seed, synth.bond_sector_chain(cfg, nr), nr, envmod.SIDE_MPS_R)
    sites = synth.site_states(synth.SPATIAL_ORBITAL)
    H, dets = fci.hamiltonian_sector(h, eri, N, twoS)
    dets = np.array(dets, dtype=np.int64)
    P = np.zeros((4 ** L, n))
    for B in blocks:
        Sa, Sb = lsec[B.a][1], rsec[B.b][1]
        t1, t2 = sites[B.s1][1], sites[B.s2][1]
        for ra in range(B.rows):
            for rb in range(B.cols):
                v = np.zeros(4 ** L)
                for mL in range(-B.jL1, B.jL1 + 1, 2):
                    mR = twoS - mL
                    if abs(mR) > B.j2R:
                        continue
                    cS = cg(B.jL1, mL, B.j2R, mR, twoS, twoS)
                    if cS == 0.0:
                        continue
                    for ma in range(-Sa, Sa + 1, 2):
                        m1 = mL - ma
                        if abs(m1) > t1:
                            continue
                        cl = cg(Sa, ma, t1, m1, B.jL1, mL)
                        if cl == 0.0:
                            continue
                        left = np.kron(_ORB_SITE[(B.s1, m1)], Ls[(B.a, ra, ma)])
                        for mb in range(-Sb, Sb + 1, 2):
                            m2 = mR - mb
                            if abs(m2) > t2:
                                continue
                            cr = cg(t2, m2, Sb, mb, B.j2R, mR)
                            if cr == 0.0:
                                continue
                            right = np.kron(Rs[(B.b, rb, mb)], _ORB_SITE[(B.s2, m2)])
                            # pattern: left orbitals below the right ones
                            v += cS * cl * cr * np.kron(right, left)
                P[:, B.offset + ra + rb * B.rows] = v
    P = P[dets, :]
    return P.T @ H @ P, P
