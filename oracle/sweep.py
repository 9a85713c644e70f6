"""Two-site sweep of SU(2) spin-adapted DMRG (Sec. II) on the ab initio
Hamiltonian (orbital sites) or the spin-1/2 Heisenberg chain: at every bond the lowest eigenpair of H_eff (Davidson), the
singular value decomposition of the reduced two-site wavefunction per bond
sector, truncation to D multiplets, and the block grown by one orbital with
the kept singular vectors (renormalisation, Sec. II.C).

Oracle module (test infrastructure only).  Plain Python/NumPy, FP64.

Readings (the paper gives no sweep algorithm):
* The reduced wavefunction across the bond between the two sites, for the
  block that grows: moving right, one matrix per left sector (N_L1, j_L1)
  with rows (left sector a, site s1) and columns (site s2, right sector b)
  of every j_2R that couples with j_L1 to the target S, j_2R ascending (the
  coupled states [(a s1)_jL1 x (s2 b)_j2R]^S are orthonormal, so its
  singular values carry the weights of the left multiplets); moving left,
  one matrix per right sector (N_2R, j_2R), rows concatenated over j_L1.
  Stacks as in ``env.mps_tensor`` (previous sector outer, site state
  inner).  At S = 0, j_L1 = j_2R and each matrix is one block row/column.
* Truncation keeps the D largest sigma^2 (one per multiplet) over all
  sectors; ties go to the lower (N, 2S) sector, then the lower index.
  Singular values with sigma^2 <= 1e-24 of the total weight are never kept:
  their singular vectors are arbitrary (the wavefunction has no weight
  there), and the bond then holds the Schmidt rank when D exceeds it.
* Moving right, the left block grows with U (the left singular vectors);
  moving left, the right block grows with V.  Each Davidson starts from a
  seeded Gaussian vector, or, with ``predict``, from the wavefunction
  predicted from the previous window (below).
* Wavefunction prediction (the standard DMRG guess; the paper does not spell
  it out).  Moving right from window i, the kept part of the bond matrix is
  U_k (U_k^T M): the left factor becomes the grown block, and the rest,
  C = U_k^T M with columns (right sector b, site s2), is expanded over the
  right block's own MPS tensor, b = [s3 x r'] (rows (r', s3)), into the
  blocks (k, s2, s3, r') of window i+1 with j_L1 = j_2R = S_b.  Moving left,
  C = M V_k is expanded over the left block's tensor, a = [a'' x s0], into
  the blocks (a'', s0, s1, k) of window i-1 with j_L1 = j_2R = S_a.  The
  spins are recoupled: (j_k (s2 S_b)_j2R)_S -> ((j_k s2)_j' S_b)_S with
  (-1)^(j_k+s2+S_b+S) sqrt((2j'+1)(2j_2R+1)) {j_k s2 j'; S_b S j_2R}, and
  moving left ((S_a s1)_jL1 j_k)_S -> (S_a (s1 j_k)_j'')_S likewise; at
  S = 0 the only term has j' = S_b (j'' = S_a) and the factor is exactly 1
  (closed form of a 6j with a zero entry).  No operator is reordered, so
  there is no fermionic sign.  The predicted vector is the
  truncated state itself, written in the next window's basis: its norm is
  sqrt(1 - discarded weight) and its Rayleigh quotient in the next window
  equals that of the truncated state in the window it came from.  At a turn
  the next window is the same one and the guess is the previous vector.
* Sweep order: bonds i = 0 .. L-2 (window sites i, i+1) left to right, then
  L-2 .. 0; the initial right blocks come from the seeded MPS of the bond
  recipe.

Parity: pinned by full CI and exact diagonalisation (with bonds that keep
every multiplet every step's energy is the ground-state energy) and by the
variational bound with truncated bonds; the prediction by the identities of
the truncated state it represents.
"""
from __future__ import annotations

import numpy as np

import synth
from . import abinitio, davidson, heff, model, sectors
from . import env as envmod
from .su2 import sixj, triangle


def _stacks(prev, sites, Nq, Sq):
    """Stacked rows (prev sector, site state) of a new sector, in the order of
    ``env.mps_tensor``: [(qp, s, r0, d)] and the total."""
    rows, r0 = [], 0
    for qp, (Np, Sp, dp) in enumerate(prev):
        for s, (ns, ts) in enumerate(sites):
            if Np + ns == Nq and triangle(Sp, ts, Sq):
                rows.append((qp, s, r0, dp))
                r0 += dp
    return rows, r0


def _bond_matrices(psi, blocks, left, right, site_kind, N, twoS=0, side="L"):
    """The two-site wavefunction across the bond between the two sites, one
    matrix per sector of the block that grows.  side 'L' (the left block
    grows): key (N_L1, j_L1), rows the left stacks (a, s1) of that sector,
    columns the right stacks (b, s2) of every j_2R coupling with j_L1 to S,
    j_2R ascending: [(j_2R, b, s2, c0, d_b)].  side 'R': key (N_2R, j_2R),
    columns its right stacks, rows the left stacks of every j_L1, ascending:
    [(j_L1, a, s1, r0, d_a)].  Returns {key: (rows, cols, M)} with the stacks
    of the growing side in ``_stacks``' 4-tuple form.  At S = 0 both forms
    hold a single spin, j_L1 = j_2R."""
    sites = synth.site_states(site_kind)
    bidx = sectors.block_index(blocks)
    if side == "L":
        keys = sorted({(left[B.a][0] + sites[B.s1][0], B.jL1) for B in blocks})
    else:
        keys = sorted({(right[B.b][0] + sites[B.s2][0], B.j2R) for B in blocks})
    out = {}
    for key in keys:
        Nk, j = key
        own, nown = _stacks(left if side == "L" else right, sites, Nk, j)
        other, n_other = [], 0
        No = N - Nk
        for jo in range(abs(j - twoS), j + twoS + 1, 2):
            st, n = _stacks(right if side == "L" else left, sites, No, jo)
            other += [(jo, q, s_, n_other + o, d) for (q, s_, o, d) in st]
            n_other += n
        if side == "L":
            M = np.zeros((nown, n_other))
            for (a, s1, r0, da) in own:
                for (jo, b, s2, c0, db) in other:
                    i = bidx.get((a, s1, s2, b, j, jo))
                    if i is not None:
                        M[r0:r0 + da, c0:c0 + db] = sectors.block_view(psi, blocks[i])
            out[key] = (own, other, M)
        else:
            M = np.zeros((n_other, nown))
            for (jo, a, s1, r0, da) in other:
                for (b, s2, c0, db) in own:
                    i = bidx.get((a, s1, s2, b, jo, j))
                    if i is not None:
                        M[r0:r0 + da, c0:c0 + db] = sectors.block_view(psi, blocks[i])
            out[key] = (other, own, M)
    return out


ZERO_WEIGHT = 1e-24


def _truncate(svals, D):
    """Indices kept per sector: the D largest sigma^2, ties to the lower
    (N, 2S) sector and then the lower index; sigma^2 at or below
    ZERO_WEIGHT times the total weight are never kept (their singular vectors
    are arbitrary)."""
    total = sum(float(np.sum(s * s)) for s in svals.values())
    cand = []
    for key, s in svals.items():
        for i, x in enumerate(s):
            if x * x > ZERO_WEIGHT * total:
                cand.append((-x * x, key, i))
    cand.sort()
    keep = {}
    for (_, key, i) in cand[:D]:
        keep.setdefault(key, []).append(i)
    return keep


def isometry(psi, blocks, left, right, site_kind, N, D, side, with_rest=False, twoS=0):
    """New bond sectors and MPS tensor of the grown block (side 'L': the left
    block grows by site 1 with U; 'R': the right block grows by site 2 with
    V), and the discarded weight.  With ``with_rest`` also the rest of the
    kept wavefunction per new sector: side 'L': (column stacks (j_2R, b, s2,
    c0, d)), U_k^T M); side 'R': (row stacks (j_L1, a, s1, r0, d), M V_k)."""
    mats = _bond_matrices(psi, blocks, left, right, site_kind, N, twoS, side)
    svd, svals = {}, {}
    for key, (lrows, rrows, M) in mats.items():
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        svd[key] = (U, Vt.T)
        svals[key] = s
    keep = _truncate(svals, D)
    # discarded weight: the sigma^2 not kept, summed directly
    dropped = sum(float(np.sum(np.delete(s, keep.get(k, [])) ** 2)) for k, s in svals.items())
    new = []
    for (Nk, j), idx in keep.items():
        new.append((Nk, j, len(idx), (Nk, j), idx))
    new.sort()
    sec = [(Nb, j, d) for (Nb, j, d, _, _) in new]
    A, rest = {}, {}
    for qo, (Nb, j, d, key, idx) in enumerate(new):
        lrows, rrows, M = mats[key]
        U, V = svd[key]
        if side == "L":
            Uk = U[:, sorted(idx)]
            A[qo] = (lrows, Uk)
            rest[qo] = (rrows, Uk.T @ M)
        else:
            Vk = V[:, sorted(idx)]
            A[qo] = (rrows, Vk)
            rest[qo] = (lrows, M @ Vk)
    if with_rest:
        return sec, A, dropped, rest
    return sec, A, dropped


def _recouple(j1, j2, j3, J, j12, j23):
    """<((j1 j2) j12, j3) J | (j1, (j2 j3) j23) J> (twos arguments): the 6j
    recoupling of three spins, (-1)^(j1+j2+j3+J) sqrt((2j12+1)(2j23+1))
    {j1 j2 j12; j3 J j23}; 1 when J = 0."""
    if J == 0:
        return 1.0 if (j12 == j3 and j23 == j1) else 0.0
    sg = -1.0 if ((j1 + j2 + j3 + J) // 2) % 2 else 1.0
    return sg * np.sqrt((j12 + 1) * (j23 + 1)) * sixj(j1, j2, j12, j3, J, j23)


def predict_moving_right(rest, right, RA, next_blocks, next_n, left_next=None, twoS=0, site_kind=None):
    """Start vector of window i+1 after the left block grew at window i:
    rest = isometry(..., 'L', with_rest=True)[3]; right = the right sectors
    of window i; RA = the MPS tensor of that right block ({b: (rows
    [(r', s3, r0, d)], G)}, rows stacked (r', s3)); left_next = the grown
    left block's sectors (needed for S > 0).  The kept wavefunction
    [k x (s2 x b)_j2R]^S, b = [s3 x r']^Sb, is recoupled to
    [(k x s2)_j' x (s3 x r')_Sb]^S."""
    out = np.zeros(next_n)
    bidx = sectors.block_index(next_blocks)
    sites = synth.site_states(site_kind) if site_kind is not None else None
    for qo, (rcols, C) in rest.items():
        jk = left_next[qo][1] if left_next is not None else None
        for (j2R, b, s2, c0, db) in rcols:
            Sb = right[b][1]
            rows_b, G = RA[b]
            X = None
            for (rp, s3, r0, drp) in rows_b:
                if twoS == 0:
                    terms = [(Sb, 1.0)]
                else:
                    t2 = sites[s2][1]
                    terms = [(jp, _recouple(jk, t2, Sb, twoS, jp, j2R))
                             for jp in range(abs(jk - t2), jk + t2 + 1, 2) if triangle(jp, Sb, twoS)]
                for (jp, w) in terms:
                    if w == 0.0:
                        continue
                    i = bidx[(qo, s2, s3, rp, jp, Sb)]
                    if X is None:
                        X = C[:, c0:c0 + db]
                    sectors.block_view(out, next_blocks[i])[:] += w * (X @ G[r0:r0 + drp, :].T)
    return out


def predict_moving_left(rest, left, LA, next_blocks, next_n, right_next=None, twoS=0, site_kind=None):
    """Start vector of window i-1 after the right block grew at window i:
    rest = isometry(..., 'R', with_rest=True)[3]; left = the left sectors of
    window i; LA = the MPS tensor of that left block ({a: (rows
    [(a'', s0, r0, d)], G)}); right_next = the grown right block's sectors
    (needed for S > 0).  [(a x s1)_jL1 x k]^S, a = [a'' x s0]^Sa, is
    recoupled to [(a'' x s0)_Sa x (s1 x k)_j'']^S."""
    out = np.zeros(next_n)
    bidx = sectors.block_index(next_blocks)
    sites = synth.site_states(site_kind) if site_kind is not None else None
    for qo, (lrows, C) in rest.items():
        jk = right_next[qo][1] if right_next is not None else None
        for (jL1, a, s1, c0, da) in lrows:
            Sa = left[a][1]
            rows_a, G = LA[a]
            for (app, s0, r0, dapp) in rows_a:
                if twoS == 0:
                    terms = [(Sa, 1.0)]
                else:
                    t1 = sites[s1][1]
                    terms = [(jpp, _recouple(Sa, t1, jk, twoS, jL1, jpp))
                             for jpp in range(abs(t1 - jk), t1 + jk + 1, 2) if triangle(Sa, jpp, twoS)]
                for (jpp, w) in terms:
                    if w == 0.0:
                        continue
                    i = bidx[(app, s0, s1, qo, Sa, jpp)]
                    sectors.block_view(out, next_blocks[i])[:] += w * (G[r0:r0 + dapp, :] @ C[c0:c0 + da, :])
    return out


def window(strings, Lb, Rb, N, twoS=0):
    """The two-site problem between blocks Lb and Rb: (apply, diag, blocks,
    psi length, left sectors, right sectors)."""
    table, env, ls, rs = abinitio.problem_from_blocks(strings, Lb, Rb)
    blocks, n = sectors.build_blocks(ls, rs, synth.SPATIAL_ORBITAL, N, twoS)
    tasks = heff.build_tasks(table, ls, rs, blocks, twoS)
    apply = lambda v: heff.apply_heff(table, env, tasks, blocks, n, v)
    diag = heff.diag_heff(table, env, tasks, blocks, n)
    return apply, diag, blocks, n, ls, rs


class HeisenbergBlock:
    """Operators {H, S} of a block of spin-1/2 sites (None for the empty
    block) on its bond sectors; grown one site at a time (the left block by
    [block x site], the right block by [site x block], Sec. II.C)."""

    def __init__(self, sectors_, H=None, S=None, J=1.0):
        self.sectors, self.H, self.S, self.J = sectors_, H, S, J

    def grown(self, cur, A, left):
        H, S = envmod.heisenberg_step(self.sectors, cur, A, self.H, self.S, left, self.J)
        return HeisenbergBlock(cur, H, S, self.J)


def heisenberg_window(Lb, Rb, N, J=1.0, twoS=0):
    """The two-site problem of the spin-1/2 Heisenberg chain between blocks
    Lb and Rb: (apply, diag, blocks, psi length, left sectors, right
    sectors)."""
    table = model.heisenberg_table(J)
    env = {}
    for side, b, ops in (("L", Lb, table.left_ops), ("R", Rb, table.right_ops)):
        for oid, op in enumerate(ops):
            if op.kind != model.MPS_RENORM:
                continue
            vals = (b.H if op.name == "H" else b.S) or {}
            env[(side, oid)] = {(qo, qi): vals.get((qo, qi), np.zeros((b.sectors[qo][2], b.sectors[qi][2])))
                                for (qo, qi) in envmod.allowed_blocks(op, b.sectors)}
    ls, rs = Lb.sectors, Rb.sectors
    blocks, n = sectors.build_blocks(ls, rs, synth.SPIN_HALF, N, twoS)
    tasks = heff.build_tasks(table, ls, rs, blocks, twoS)
    apply = lambda v: heff.apply_heff(table, env, tasks, blocks, n, v)
    diag = heff.diag_heff(table, env, tasks, blocks, n)
    return apply, diag, blocks, n, ls, rs


def _solve(win, seed, tol, x0=None):
    apply, diag, blocks, n, ls, rs = win
    if x0 is None or not np.linalg.norm(x0) > 0:
        x0 = synth.gaussian_psi(n, seed)
    rq0 = float(x0 @ apply(x0) / (x0 @ x0))
    theta, x, res, it = davidson.davidson(apply, diag, x0, tol=tol)
    return theta, x, blocks, ls, rs, it, rq0


def sweep(cfg, D, n_half, tol=1e-9, h=None, eri=None, predict=False, stats=None, J=1.0):
    """Energies of every two-site step of n_half half-sweeps (target spin
    cfg.twoS / 2), with the
    initial right blocks from cfg's seeded MPS; returns (energies, discarded
    weights).  The model follows cfg's site kind: the ab initio Hamiltonian
    of the integrals (h, eri; default: cfg's seeded ones) on orbital sites,
    or the Heisenberg chain with coupling J on spin-1/2 sites.  With
    ``predict`` every window after the first starts from the wavefunction
    predicted from the previous one.  A list ``stats`` receives (Davidson
    iterations, Rayleigh quotient of the start vector) per step."""
    kind = cfg.site_kind
    L, N, twoS = cfg.L, cfg.N, cfg.twoS
    if kind == synth.SPATIAL_ORBITAL:
        if h is None:
            h, eri = synth.integrals(cfg.L, cfg.seed)
        strings = abinitio.hamiltonian_strings(h, eri)
        R = [abinitio.RightBlock(strings, L)]
        Lbs = [abinitio.LeftBlock(strings, L)] + [None] * (L - 2)
        grow = lambda b, sec, A, left: b.grown(sec, A)
        make_window = lambda Lb, Rb: window(strings, Lb, Rb, N, twoS)
    else:
        R = [HeisenbergBlock([(0, 0, 1)], J=J)]
        Lbs = [HeisenbergBlock([(0, 0, 1)], J=J)] + [None] * (L - 2)
        grow = lambda b, sec, A, left: b.grown(sec, A, left)
        make_window = lambda Lb, Rb: heisenberg_window(Lb, Rb, N, J, twoS)
    chain = synth.bond_sector_chain(cfg, L - 2)
    # R[m]: right block of the last m sites; RA[m] / LA[m]: the MPS tensor
    # that grew R[m] from R[m-1] / Lbs[m] from Lbs[m-1]
    RA = [None] * (L - 1)
    for k in range(1, L - 1):
        A = envmod.mps_tensor(cfg.seed, envmod.SIDE_MPS_R, k, chain[k - 1], chain[k], kind)
        R.append(grow(R[-1], chain[k], A, False))
        RA[k] = A
    LA = [None] * (L - 1)
    energies, discarded = [], []
    step = 0
    guess = None
    for half in range(n_half):
        order = range(0, L - 1) if half % 2 == 0 else range(L - 2, -1, -1)
        for i in order:
            Lb, Rb = Lbs[i], R[L - 2 - i]
            theta, x, blocks, ls, rs, it, rq0 = _solve(make_window(Lb, Rb), cfg.seed + 1000 + step, tol,
                                                       guess if predict else None)
            if stats is not None:
                stats.append((it, rq0))
            step += 1
            energies.append(theta)
            guess = x   # at a turn the next window is this one
            if half % 2 == 0 and i < L - 2:
                sec, A, w, rest = isometry(x, blocks, ls, rs, kind, N, D, "L", with_rest=True, twoS=twoS)
                Lbs[i + 1] = grow(Lb, sec, A, True)
                LA[i + 1] = A
                discarded.append(w)
                if predict:
                    nb, nn = sectors.build_blocks(Lbs[i + 1].sectors, R[L - 3 - i].sectors, kind, N, twoS)
                    guess = predict_moving_right(rest, rs, RA[L - 2 - i], nb, nn, sec, twoS, kind)
            elif half % 2 == 1 and i > 0:
                sec, A, w, rest = isometry(x, blocks, ls, rs, kind, N, D, "R", with_rest=True, twoS=twoS)
                R[L - 1 - i] = grow(Rb, sec, A, False)
                RA[L - 1 - i] = A
                discarded.append(w)
                if predict:
                    nb, nn = sectors.build_blocks(Lbs[i - 1].sectors, R[L - 1 - i].sectors, kind, N, twoS)
                    guess = predict_moving_left(rest, ls, LA[i], nb, nn, sec, twoS, kind)
    return np.array(energies), np.array(discarded)
