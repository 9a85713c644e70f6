"""Block operators A_i (left) and D_i (right) at the two-site bond.

Oracle module (test infrastructure only).

* Synthetic-entry operators (ab initio skeleton): every allowed sector block
  (N' = N + dN, triangle(S, k, S')) of a RANDOM operator is filled from a
  counter-based generator, SplitMix64 (Steele, Lea, Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): the stream of a block is
  seeded by chaining the SplitMix64 output function over
  (seed, side, op id, (out sector << 32) | in sector), and element idx
  (column-major) is mix64(key + (idx+1)*gamma) mapped to [-1, 1) by
  (x >> 11) * 2^-53 * 2 - 1, then scaled by 1/sqrt(max(d_out, d_in)).
  HAM blocks (q,q): 0.1*(X + X^T) + diag(2 r / d_q).  ADJOINT operators use
  the adjoint-tensor rule of ``model.adjoint_reduced``.
* Heisenberg block operators (H_block and the edge spin S) are renormalised
  from a seeded SU(2) MPS, block x site with the W9j^(l) factor on the left
  and site x block with W9j^(r) on the right (Sec. II.C); each MPS tensor is
  the Q factor (positive diagonal of R) of a counter-generated Gaussian-free
  uniform matrix stacked over the (previous sector, site state) pairs.

Parity: the Heisenberg operators are pinned by the explicit full-space
projection in ``expand`` and by exact diagonalisation; synthetic operators
enter only through H.psi, pinned by the m-resolved expansion.
"""
from __future__ import annotations

import math

import numpy as np

import synth
from . import model
from .model import ADJOINT, HAM, IDENTITY, MPS_RENORM, NUMTOT, RANDOM, SPINTOT
from .su2 import ctilde, triangle

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    """SplitMix64 output function on uint64 numpy arrays (wrapping)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _mix_int(x: int) -> int:
    x &= MASK
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & MASK
    return x ^ (x >> 31)


def splitmix(x: int) -> int:
    return _mix_int((x + GAMMA) & MASK)


def block_key(seed, side, op, q_out, q_in) -> int:
    h = splitmix(seed)
    h = splitmix(h ^ side)
    h = splitmix(h ^ op)
    return splitmix(h ^ ((q_out << 32) | q_in))


def uniform_block(key: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols matrix, column-major element stream, values in [-1, 1)."""
    n = rows * cols
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = mix64(np.uint64(key) + idx * np.uint64(GAMMA))
    u = (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
    return u.reshape(cols, rows).T


SIDE_L, SIDE_R, SIDE_MPS_L, SIDE_MPS_R = 0, 1, 2, 3


def allowed_blocks(op, sectors):
    res = []
    for qi, (Ni, Si, _) in enumerate(sectors):
        for qo, (No, So, _) in enumerate(sectors):
            if No == Ni + op.dN and triangle(Si, op.k, So):
                res.append((qo, qi))
    return res


def synthetic_ops(table, sectors, side_name, seed):
    """Values of all non-identity operators of one side, synthetic entries."""
    side = SIDE_L if side_name == "L" else SIDE_R
    ops = table.left_ops if side_name == "L" else table.right_ops
    out = {}
    for oid, op in enumerate(ops):
        if op.kind == RANDOM:
            blk = {}
            for (qo, qi) in allowed_blocks(op, sectors):
                do, di = sectors[qo][2], sectors[qi][2]
                s = 1.0 / math.sqrt(max(do, di))
                blk[(qo, qi)] = uniform_block(block_key(seed, side, oid, qo, qi), do, di) * s
            out[oid] = blk
        elif op.kind == HAM:
            blk = {}
            for q, (_, _, d) in enumerate(sectors):
                s = 1.0 / math.sqrt(d)
                X = uniform_block(block_key(seed, side, oid, q, q), d, d) * s
                H = 0.1 * (X + X.T)
                H[np.diag_indices(d)] += (2.0 * np.arange(d)) / d
                blk[(q, q)] = H
            out[oid] = blk
    for oid, op in enumerate(ops):
        if op.kind == ADJOINT:
            out[oid] = adjoint_blocks(out[op.base], ops[op.base].k, sectors)
    return out


def adjoint_blocks(blocks, k, sectors):
    """Adjoint tensor: block (a,b) = (-1)^{(S_b+k-S_a)/2} sqrt((S_b+1)/(S_a+1)) T(b,a)^T."""
    res = {}
    for (qo, qi), M in blocks.items():
        Sa, Sb = sectors[qi][1], sectors[qo][1]      # new out = old in (a), new in = old out (b)
        e = Sb + k - Sa
        assert e % 2 == 0
        sign = -1.0 if (e // 2) % 2 else 1.0
        res[(qi, qo)] = sign * math.sqrt((Sb + 1) / (Sa + 1)) * M.T
    return res


# ---------------------------------------------------------------------------
# seeded MPS and Heisenberg renormalisation

def mps_tensor(seed, mps_side, site, prev, cur, site_kind):
    """MPS tensor from bond ``prev`` to bond ``cur`` (sector lists).

    Returns {q_out: (rows list [(q_prev, sigma, row0, d)], Q matrix)} where
    the stacked rows run over (q_prev ascending, sigma ascending) pairs that
    couple to q_out, and Q has orthonormal columns (Gram-Schmidt orientation).
    """
    sites = synth.site_states(site_kind)
    res = {}
    for qo, (No, So, do) in enumerate(cur):
        rows = []
        r0 = 0
        for qp, (Np, Sp, dp) in enumerate(prev):
            for s, (ns, ts) in enumerate(sites):
                if Np + ns == No and triangle(Sp, ts, So):
                    rows.append((qp, s, r0, dp))
                    r0 += dp
        if r0 < do:
            raise ValueError("bond dimension exceeds the available states")
        G = uniform_block(block_key(seed, mps_side, site, qo, 0), r0, do)
        Q, R = np.linalg.qr(G)
        sg = np.sign(np.diag(R))
        sg[sg == 0] = 1.0
        res[qo] = (rows, Q * sg)
    return res


def _coupled_op(prev, sites, T, rows_o, rows_i, Sout, Sin, blockop, kO, pO, siteop, left_side, K):
    """Reduced matrix of [O x s]^K (left) or [s x O]^K (right) between
    stacked coupled rows (out rows x in rows)."""
    sm = siteop.mat()
    M = np.zeros((rows_o[-1][2] + rows_o[-1][3] if rows_o else 0,
                  rows_i[-1][2] + rows_i[-1][3] if rows_i else 0))
    for (qpo, so, ro, dpo) in rows_o:
        for (qpi, si, ri, dpi) in rows_i:
            sv = sm[so, si]
            if sv == 0.0:
                continue
            if blockop is None:                     # identity on the block
                if qpo != qpi:
                    continue
                Ob = np.eye(dpo)
            else:
                Ob = blockop.get((qpo, qpi))
                if Ob is None:
                    continue
            Sl_i, Sl_o = prev[qpi][1], prev[qpo][1]
            ts_i, ts_o = sites[si][1], sites[so][1]
            if left_side:
                c = ctilde(Sl_i, ts_i, Sin, kO, siteop.k, K, Sl_o, ts_o, Sout)
                sgn = -1.0 if (siteop.parity * (prev[qpi][0] % 2)) else 1.0
            else:
                c = ctilde(ts_i, Sl_i, Sin, siteop.k, kO, K, ts_o, Sl_o, Sout)
                sgn = -1.0 if (pO * (sites[si][0] % 2)) else 1.0
            if c == 0.0:
                continue
            M[ro:ro + dpo, ri:ri + dpi] += sgn * c * sv * Ob
    return M


def heisenberg_block_ops(cfg, n_sites, mps_side, J=1.0):
    """Renormalised {H, S} of a block of ``n_sites`` spin-1/2 sites.

    Left block: H' = [H x 1]^0 - sqrt(3) J [S x s]^0, S' = [1 x s]^1.
    Right block (site added on the left): H' = [1 x H]^0 - sqrt(3) J [s x S]^0,
    S' = [s x 1]^1.  Returns (sectors, {'H': blocks, 'S': blocks}).
    """
    sk = synth.SPIN_HALF
    chain = synth.bond_sector_chain(cfg, n_sites)
    left = mps_side == SIDE_MPS_L
    H, S = None, None
    for k in range(1, n_sites + 1):
        A = mps_tensor(cfg.seed, mps_side, k, chain[k - 1], chain[k], sk)
        H, S = heisenberg_step(chain[k - 1], chain[k], A, H, S, left, J)
    return chain[n_sites], {"H": H, "S": S}


def heisenberg_step(prev, cur, A, H, S, left, J=1.0):
    """One growth step of a Heisenberg block by a spin-1/2 site: the block's
    {H, S} on bond ``prev`` (None for the empty block) projected by the MPS
    tensor A (``mps_tensor``'s layout) onto bond ``cur``."""
    sites = synth.site_states(synth.SPIN_HALF)
    so = model.site_ops(synth.SPIN_HALF)
    Hn, Sn = {}, {}
    for qo, (rows_o, Qo) in A.items():
        for qi, (rows_i, Qi) in A.items():
            So_, Si_ = cur[qo][1], cur[qi][1]
            if cur[qo][0] != cur[qi][0]:
                continue
            if So_ == Si_:
                M = np.zeros((Qo.shape[0], Qi.shape[0]))
                if H is not None:
                    M += _coupled_op(prev, sites, None, rows_o, rows_i, So_, Si_, H, 0, 0,
                                     so["I"], left, 0)
                if S is not None:
                    M += -math.sqrt(3.0) * J * _coupled_op(prev, sites, None, rows_o, rows_i,
                                                           So_, Si_, S, 2, 0, so["S"], left, 0)
                Hn[(qo, qi)] = Qo.T @ M @ Qi
            if triangle(Si_, 2, So_):
                M = _coupled_op(prev, sites, None, rows_o, rows_i, So_, Si_, None, 0, 0,
                                so["S"], left, 2)
                Sn[(qo, qi)] = Qo.T @ M @ Qi
    return Hn, Sn


def casimir_ops(table, sectors, side_name):
    """Block total spin (name 'S': sqrt(S(S+1)) per sector; 'S2': S(S+1))
    and particle number (N) as reduced blocks: diagonal in the sector, zero
    blocks for the other structurally allowed sector pairs."""
    ops = table.left_ops if side_name == "L" else table.right_ops
    out = {}
    for oid, op in enumerate(ops):
        if op.kind not in (SPINTOT, NUMTOT):
            continue
        blk = {}
        for (qo, qi) in allowed_blocks(op, sectors):
            N, S, d = sectors[qi]
            M = np.zeros((sectors[qo][2], d))
            if qo == qi:
                j = S / 2.0
                if op.kind == NUMTOT:
                    val = float(N)
                elif op.name == "S2":
                    val = j * (j + 1)
                else:
                    val = math.sqrt(j * (j + 1))
                M = val * np.eye(d)
            blk[(qo, qi)] = M
        out[oid] = blk
    return out


def build_env(table, cfg, left, right):
    """(side, op id) -> blocks for every non-identity operator of ``table``."""
    env = {}
    if any(op.kind in (SPINTOT, NUMTOT) for op in table.left_ops + table.right_ops):
        for side, sectors in (("L", left), ("R", right)):
            for oid, blk in casimir_ops(table, sectors, side).items():
                env[(side, oid)] = blk
        return env
    if cfg.site_kind == synth.SPIN_HALF:
        lsec, lops = heisenberg_block_ops(cfg, cfg.n_left, SIDE_MPS_L)
        rsec, rops = heisenberg_block_ops(cfg, cfg.n_right, SIDE_MPS_R)
        assert lsec == left and rsec == right
        for side, ops, vals in (("L", table.left_ops, lops), ("R", table.right_ops, rops)):
            for oid, op in enumerate(ops):
                if op.kind == MPS_RENORM:
                    env[(side, oid)] = vals[op.name]
        return env
    for side, sectors in (("L", left), ("R", right)):
        for oid, blk in synthetic_ops(table, sectors, side, cfg.seed).items():
            env[(side, oid)] = blk
    return env


class _LazyOp:
    def __init__(self, owner, side, oid):
        self.owner, self.side, self.oid = owner, side, oid
        self.cache = {}

    def __getitem__(self, key):
        if key not in self.cache:
            self.cache[key] = self.owner.block(self.side, self.oid, key)
        return self.cache[key]


class LazySyntheticEnv:
    """Synthetic-entry operators computed block by block on demand (same
    values as ``synthetic_ops``), for sampled checks of large problems."""

    def __init__(self, table, cfg, left, right):
        self.table, self.cfg = table, cfg
        self.sectors = {"L": left, "R": right}
        self.ops = {"L": table.left_ops, "R": table.right_ops}
        self._lazy = {}

    def __getitem__(self, key):
        if key not in self._lazy:
            self._lazy[key] = _LazyOp(self, *key)
        return self._lazy[key]

    def get(self, key, default=None):
        return self[key]

    def block(self, side, oid, key):
        qo, qi = key
        op = self.ops[side][oid]
        sec = self.sectors[side]
        sid = SIDE_L if side == "L" else SIDE_R
        if op.kind == RANDOM:
            if not (sec[qo][0] == sec[qi][0] + op.dN and triangle(sec[qi][1], op.k, sec[qo][1])):
                raise KeyError(key)
            do, di = sec[qo][2], sec[qi][2]
            s = 1.0 / math.sqrt(max(do, di))
            return uniform_block(block_key(self.cfg.seed, sid, oid, qo, qi), do, di) * s
        if op.kind == HAM:
            if qo != qi:
                raise KeyError(key)
            d = sec[qo][2]
            s = 1.0 / math.sqrt(d)
            X = uniform_block(block_key(self.cfg.seed, sid, oid, qo, qo), d, d) * s
            H = 0.1 * (X + X.T)
            H[np.diag_indices(d)] += (2.0 * np.arange(d)) / d
            return H
        if op.kind == ADJOINT:
            base = self[(side, op.base)][(qi, qo)]
            k = self.ops[side][op.base].k
            Sa, Sb = sec[qo][1], sec[qi][1]
            e = Sb + k - Sa
            sign = -1.0 if (e // 2) % 2 else 1.0
            return sign * math.sqrt((Sb + 1) / (Sa + 1)) * base.T
        raise KeyError(key)
