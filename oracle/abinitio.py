"""Ab initio Hamiltonian (Eq. 1) at a two-site bond: spin-adapted block
operators in the normal/complementary partition (Sec. II.A), renormalised
from a seeded SU(2) MPS with the W9j^(l) / W9j^(r) factors (Sec. II.C), and
the operator-table of Eq. 2 built from them.

Oracle module (test infrastructure only).  Plain Python/NumPy, FP64.

Reading of the paper (it states the precontracted operators of Sec. II.A but
not their spin-adapted form):

* H = sum_ij h_ij sum_s c+_is c_js + 1/2 sum_ijkl (ij|kl) sum_st c+_is c+_kt
  c_lt c_js.  Every term is written as a product of elementary rank-1/2
  tensors, the creator a+_i (a+_m = c+_{i,m}) and the annihilator tensor
  a~_i (a~_{+1/2} = c_{i,dn}, a~_{-1/2} = -c_{i,up}), put in Jordan-Wigner
  order (orbital, creators first) with the sign of the permutation.  A
  "string" is such an ordered product; its coefficients over the spin
  components form a formal tensor F_S (all integral terms with the same
  ordered operator list are summed into one F_S).
* Spin coupling is done numerically: a coupled product is a binary tree of
  Clebsch-Gordan couplings; the coefficient of a string on a coupled basis
  element is the overlap of the two component tensors (the coupled bases are
  orthonormal).  Recoupling coefficients between two trees over the same
  leaves are overlaps as well.
* Right block (orbitals after the two sites): complementary operators.  For a
  set O of elementary operators outside the block (left-nested coupling
  labels lam, rank k), C(O, lam) = sum over strings S whose outside part is
  O of the block part of S, so that H = sum_O [O^lam x C(O, lam)]^0.  Stored
  for |O| <= 2 (|O| = 0 is the block Hamiltonian); |O| = 3 is a combination
  of the block's elementary operators, |O| = 4 a number.  Growing the block
  by a site s: C'(O', lam') = sum over strings Y on s of W [Y x C(O' + Y)],
  W the recoupling overlap (Sec. II.C's W9j^(r) then couples site x block).
* Left block (orbitals before the two sites): normal operators with one and
  two elementary factors, and complementary operators with |O| <= 1 (the
  block Hamiltonian and the three-index operators S(o)).
* Middle bond: every string is assigned to exactly one family of rows of
  Eq. 2 (left complementary x sites x right normal, left normal x sites x
  right complementary, or sites only), so that the rows sum to H.
* Fermion signs: Jordan-Wigner order L, s1, s2, R (as in ``heff``).

Parity: pinned by full configuration interaction (``fci``): with bond
dimensions that keep every multiplet, the spectrum of the SU(2) H_eff equals
the spin-S part of the N-electron spectrum of H; and by Hermiticity of H_eff
with truncated bonds.
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np

import synth
from . import env as envmod
from . import model
from .su2 import cg, ctilde, triangle

# ---------------------------------------------------------------------------
# elementary tensors and the Hamiltonian as formal tensors

CREATE, ANNIHILATE = 1, 0


def canon_key(op):
    return (op[0], 1 - op[1])


def _perm_sign(order):
    sign, seen = 1, [False] * len(order)
    for i in range(len(order)):
        if seen[i]:
            continue
        j, n = i, 0
        while not seen[j]:
            seen[j] = True
            j = order[j]
            n += 1
        if n % 2 == 0:
            sign = -sign
    return sign


def _one_body_tensor():
    """sum_s c+_s c_s over the components of (a+, a~): c_up = -a~_{-1/2},
    c_dn = a~_{+1/2}; component index 0 is m = +1/2, 1 is m = -1/2."""
    F = np.zeros((2, 2))
    for s in (0, 1):
        F[s, 1 - s] = -1.0 if s == 0 else 1.0
    return F


def _two_body_tensor():
    """sum_st c+_s c+_t c_t c_s over the components of (a+, a+, a~, a~)."""
    F = np.zeros((2, 2, 2, 2))
    for s in (0, 1):
        for t in (0, 1):
            F[s, t, 1 - t, 1 - s] = (-1.0 if t == 0 else 1.0) * (-1.0 if s == 0 else 1.0)
    return F


def hamiltonian_strings(h, eri, tol=0.0):
    """{string (tuple of (orbital, dag)) : F_S}: the Hamiltonian as a sum of
    ordered products of elementary tensors with formal component tensors."""
    L = h.shape[0]
    out = {}
    F1, F2 = _one_body_tensor(), _two_body_tensor()

    def add(ops, F):
        order = sorted(range(len(ops)), key=lambda a: canon_key(ops[a]))
        key = tuple(ops[a] for a in order)
        G = np.transpose(F, order) * _perm_sign(order)
        if key in out:
            out[key] = out[key] + G
        else:
            out[key] = G

    for i in range(L):
        for j in range(L):
            if abs(h[i, j]) > tol:
                add([(i, CREATE), (j, ANNIHILATE)], h[i, j] * F1)
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = eri[i, j, k, l]
                    if abs(v) > tol:
                        add([(i, CREATE), (k, CREATE), (l, ANNIHILATE), (j, ANNIHILATE)], 0.5 * v * F2)
    return out


# ---------------------------------------------------------------------------
# coupling trees: ('e',) an elementary rank-1/2 leaf, ('x', j) a leaf of rank
# j (twos), ('0',) the empty (scalar) leaf, ('n', left, right, K) the coupling
# of left and right to rank K.  In-order leaves are the tensor axes.

E = ("e",)
ZERO = ("0",)


@lru_cache(maxsize=None)
def _tree(t):
    kind = t[0]
    if kind == "e":
        return {1: np.array([1.0, 0.0]), -1: np.array([0.0, 1.0])}, 1
    if kind == "0":
        return {0: np.array([1.0])}, 0
    if kind == "x":
        j = t[1]
        d = {}
        for idx, m in enumerate(range(j, -j - 1, -2)):
            v = np.zeros(j + 1)
            v[idx] = 1.0
            d[m] = v
        return d, j
    _, l, r, K = t
    dl, jl = _tree(l)
    dr, jr = _tree(r)
    res = {}
    for ml, vl in dl.items():
        for mr, vr in dr.items():
            M = ml + mr
            if abs(M) > K:
                continue
            c = cg(jl, ml, jr, mr, K, M)
            if c != 0.0:
                x = c * np.multiply.outer(vl, vr)
                res[M] = res[M] + x if M in res else x
    return res, K


def rank_of(t):
    return _tree(t)[1]


@lru_cache(maxsize=None)
def overlap(t1, t2):
    """<t1|t2> of two rank-0 trees over the same leaves (size-1 axes dropped)."""
    v1 = _tree(t1)[0].get(0)
    v2 = _tree(t2)[0].get(0)
    if v1 is None or v2 is None:
        return 0.0
    a, b = np.squeeze(v1), np.squeeze(v2)
    assert a.shape == b.shape, (t1, t2)
    return float(np.sum(a * b))


def lnest(n, labels):
    """Left-nested coupling of n elementary leaves with intermediate ranks."""
    if n == 0:
        return ZERO
    t = E
    for i in range(1, n):
        t = ("n", t, E, labels[i - 1])
    return t


@lru_cache(maxsize=None)
def labelings(n):
    """All intermediate-rank tuples of a left-nested coupling of n spin-1/2."""
    if n <= 1:
        return [()]
    res = []
    for lab in labelings(n - 1):
        j = lab[-1] if lab else 1
        for K in range(abs(j - 1), j + 2, 2):
            res.append(lab + (K,))
    return res


def lab_rank(n, lab):
    return 0 if n == 0 else (1 if n == 1 else lab[-1])


def string_coef(tree, F):
    """Coefficient of the formal tensor F on a rank-0 coupled basis element."""
    v = _tree(tree)[0].get(0)
    if v is None:
        return 0.0
    return float(np.sum(np.squeeze(v) * F))


def valid_labels(ops, lab):
    """Drop couplings that vanish identically: two equal elementary operators
    coupled directly to rank 1 ([a+_i x a+_i]^1 = 0, [a~_i x a~_i]^1 = 0)."""
    if len(ops) >= 2 and ops[0] == ops[1] and lab[0] == 2:
        return False
    return True


# ---------------------------------------------------------------------------
# site operators of a string on one orbital

_SITE_STATES = [(0, 0, [(0, 0)]), (1, 1, [(1, 1), (-1, 2)]), (2, 0, [(0, 3)])]  # (N, 2S, [(2m, fock index)])


def _fock_site():
    cu = np.zeros((4, 4)); cd = np.zeros((4, 4))
    cu[1, 0] = 1.0; cu[3, 2] = 1.0          # c+_up |dn> = c+_up c+_dn |0> = |2>
    cd[2, 0] = 1.0; cd[3, 1] = -1.0         # c+_dn |up> = -|2>
    adag = [cu, cd]                         # component 0: m = +1/2
    atil = [cd.T.copy(), -cu.T.copy()]      # a~_{+1/2} = c_dn, a~_{-1/2} = -c_up
    return adag, atil


@lru_cache(maxsize=None)
def site_op(dags, lab):
    """Reduced 3x3 site matrix (CG form of Wigner-Eckart) of the left-nested
    coupled product of elementary tensors with the given dag flags on one
    orbital; None if it vanishes."""
    n = len(dags)
    if n == 0:
        return model.site_ops(synth.SPATIAL_ORBITAL)["I"]
    adag, atil = _fock_site()
    comps, k = _tree(lnest(n, lab))
    T = {}
    for q, v in comps.items():
        M = np.zeros((4, 4))
        for idx in np.ndindex(*v.shape):
            c = v[idx]
            if c == 0.0:
                continue
            P = np.eye(4)
            for a, d in enumerate(dags):
                P = P @ (adag[idx[a]] if d == CREATE else atil[idx[a]])
            M += c * P
        T[q] = M
    red = np.zeros((3, 3))
    for so, (No, So, mo_list) in enumerate(_SITE_STATES):
        for si, (Ni, Si, mi_list) in enumerate(_SITE_STATES):
            vals = []
            for (mo, fo) in mo_list:
                for (mi, fi) in mi_list:
                    q = mo - mi
                    if abs(q) > k or q not in T:
                        continue
                    c = cg(Si, mi, k, q, So, mo)
                    if c == 0.0:
                        continue
                    vals.append(T[q][fo, fi] / c)
            if vals:
                assert max(vals) - min(vals) <= 1e-12, vals
                red[so, si] = vals[0]
    if np.all(np.abs(red) < 1e-15):
        return None
    dN = sum(1 if d == CREATE else -1 for d in dags)
    return model.SiteOp(f"site{dags}{lab}", k, dN, n % 2, model._tup(red))


def site_strings(max_len):
    """Canonical strings on one orbital: creators first, at most two of each."""
    res = []
    for nc in range(3):
        for na in range(3):
            if 0 < nc + na <= max_len:
                res.append((CREATE,) * nc + (ANNIHILATE,) * na)
    return res


# ---------------------------------------------------------------------------
# block operators

class BOp:
    """Reduced block operator: rank k (twos), particle change dN, parity and
    blocks {(q_out, q_in): matrix}."""

    def __init__(self, k, dN, parity, blocks):
        self.k, self.dN, self.parity, self.blocks = k, dN, parity, blocks

    def scaled_add(self, other, c):
        for key, M in other.blocks.items():
            if key in self.blocks:
                self.blocks[key] = self.blocks[key] + c * M
            else:
                self.blocks[key] = c * M


def _identity(sectors, c=1.0):
    return BOp(0, 0, 0, {(q, q): c * np.eye(d) for q, (_, _, d) in enumerate(sectors)})


def _ops_meta(ops):
    dN = sum(1 if d == CREATE else -1 for (_, d) in ops)
    return dN, len(ops) % 2


class _Grow:
    """One renormalisation step: coupled products of a site operator and an
    operator of the previous block, projected on the new bond's MPS basis."""

    def __init__(self, A, prev, cur, left):
        """A: MPS tensor {new sector: (stacked rows [(q_prev, site, row0, d)],
        Q with orthonormal columns)} from bond `prev` to bond `cur`."""
        self.left = left
        self.A = A
        self.prev, self.cur = prev, cur
        self.sites = synth.site_states(synth.SPATIAL_ORBITAL)

    def build(self, k, dN, parity, contribs):
        """contribs: list of (coef, SiteOp, BOp or None (identity), K)."""
        blocks = {}
        for qo, (rows_o, Qo) in self.A.items():
            for qi, (rows_i, Qi) in self.A.items():
                No, So, _ = self.cur[qo]
                Ni, Si, _ = self.cur[qi]
                if No != Ni + dN or not triangle(Si, k, So):
                    continue
                M = np.zeros((Qo.shape[0], Qi.shape[0]))
                for coef, Y, X, K in contribs:
                    kX = 0 if X is None else X.k
                    pX = 0 if X is None else X.parity
                    M += coef * envmod._coupled_op(self.prev, self.sites, None, rows_o, rows_i, So, Si,
                                                   None if X is None else X.blocks, kX, pX, Y, self.left, K)
                blocks[(qo, qi)] = Qo.T @ M @ Qi
        return BOp(k, dN, parity, blocks)


def _outside_keys(outside_ops, max_len):
    """Canonical outside sets O (|O| <= max_len) with their coupling labels."""
    keys = [((), ())]
    n = len(outside_ops)
    for a in range(n):
        keys.append(((outside_ops[a],), ()))
    if max_len >= 2:
        for a in range(n):
            for b in range(a, n):
                O = (outside_ops[a], outside_ops[b])
                for lab in labelings(2):
                    if valid_labels(O, lab):
                        keys.append((O, lab))
    return keys


def _elementary(orbs):
    res = []
    for o in orbs:
        res.append((o, CREATE))
        res.append((o, ANNIHILATE))
    return res


class RightBlock:
    """Operators of a right block (orbitals first .. L-1), grown from the
    vacuum one orbital at a time (site added on the left of the block)."""

    def __init__(self, strings, L):
        self.S = strings
        self.L = L
        self.sectors = [(0, 0, 1)]
        self.orbs = []
        self.N1, self.C = {}, {}
        self._direct_cache = {}

    @classmethod
    def seeded(cls, strings, cfg, n_sites):
        """The block of the last n_sites orbitals of cfg from its seeded MPS."""
        b = cls(strings, cfg.L)
        chain = synth.bond_sector_chain(cfg, n_sites)
        for step in range(1, n_sites + 1):
            A = envmod.mps_tensor(cfg.seed, envmod.SIDE_MPS_R, step, chain[step - 1], chain[step],
                                  synth.SPATIAL_ORBITAL)
            b = b.grown(chain[step], A)
        return b

    def grown(self, cur, A):
        """A new block: this one with orbital s = first - 1 added on its left,
        projected on the bond `cur` by the MPS tensor A (rows stacked
        (block sector, site state), see ``env.mps_tensor``)."""
        s = (self.orbs[0] if self.orbs else self.L) - 1
        g = _Grow(A, self.sectors, cur, left=False)
        outside = _elementary(range(s))
        N1, C = {}, {}
        I_site = site_op((), ())
        for (o, d) in _elementary([s]):
            N1[(o, d)] = g.build(1, 1 if d == CREATE else -1, 1, [(1.0, site_op((d,), ()), None, 1)])
        for x, X in self.N1.items():
            N1[x] = g.build(1, X.dN, 1, [(1.0, I_site, X, 1)])
        for (O, lam) in _outside_keys(outside, 2):
            kO = lab_rank(len(O), lam)
            dN, par = _ops_meta(O)
            contribs = self._recursion(O, lam, s)
            if contribs:
                C[(O, lam)] = g.build(kO, -dN, par, contribs)
        b = RightBlock(self.S, self.L)
        b.N1, b.C = N1, C
        b.orbs = [s] + self.orbs
        b.sectors = list(cur)
        return b

    def get(self, O, lam):
        """C(O, lam) of the current block (None when it vanishes)."""
        if len(O) <= 2 and self.orbs:
            return self.C.get((O, lam))
        return self._direct(O, lam)

    def _direct(self, O, lam):
        key = (O, lam)
        if key in self._direct_cache:
            return self._direct_cache[key]
        res = None
        n = len(O)
        if n % 2 == 0:                               # no block operator left: a number
            if lab_rank(n, lam) == 0 and O in self.S:
                c = string_coef(lnest(n, lam), self.S[O])
                if c != 0.0:
                    res = _identity(self.sectors, c)
        elif self.orbs:                              # one elementary block operator
            dN, par = _ops_meta(O)
            acc = None
            for x in _elementary(self.orbs):
                S = O + (x,)
                if S not in self.S:
                    continue
                c = string_coef(("n", lnest(n, lam), E, 0), self.S[S])
                if c == 0.0:
                    continue
                if acc is None:
                    acc = BOp(1, -dN, 1, {})
                acc.scaled_add(self.N1[x], c)
            res = acc
        self._direct_cache[key] = res
        return res

    def _recursion(self, O1, lam1, s):
        k1 = lab_rank(len(O1), lam1)
        contribs = []
        for Y in [()] + site_strings(4 - len(O1)):
            nY = len(Y)
            Yops = tuple((s, d) for d in Y)
            O = O1 + Yops
            for nu in labelings(nY):
                if nY and not valid_labels(Yops, nu):
                    continue
                Yop = site_op(Y, nu)
                if Yop is None:
                    continue
                kY = lab_rank(nY, nu)
                for lam in labelings(len(O)):
                    if not valid_labels(O, lam):
                        continue
                    kX = lab_rank(len(O), lam)
                    if not triangle(kY, kX, k1):
                        continue
                    W = overlap(("n", lnest(len(O1), lam1), ("n", lnest(nY, nu), ("x", kX), k1), 0),
                                ("n", lnest(len(O), lam), ("x", kX), 0))
                    if abs(W) < 1e-14:
                        continue
                    X = self.get(O, lam)
                    if X is None:
                        continue
                    if X.k != kX:
                        continue
                    contribs.append((W, Yop, X, k1))
        return contribs


class LeftBlock:
    """Operators of a left block (orbitals 0 .. n-1), grown from the vacuum
    one orbital at a time (site added on the right of the block): normal
    operators with one and two elementary factors, complementary operators
    with |O| <= 1 outside factors (H and the three-index operators)."""

    def __init__(self, strings, L):
        self.S = strings
        self.L = L
        self.sectors = [(0, 0, 1)]
        self.orbs = []
        self.N1, self.N2, self.C = {}, {}, {}
        self._direct_cache = {}

    @classmethod
    def seeded(cls, strings, cfg, n_sites):
        """The block of the first n_sites orbitals of cfg from its seeded MPS."""
        b = cls(strings, cfg.L)
        chain = synth.bond_sector_chain(cfg, n_sites)
        for step in range(1, n_sites + 1):
            A = envmod.mps_tensor(cfg.seed, envmod.SIDE_MPS_L, step, chain[step - 1], chain[step],
                                  synth.SPATIAL_ORBITAL)
            b = b.grown(chain[step], A)
        return b

    def grown(self, cur, A):
        """A new block: this one with orbital s = last + 1 added on its right,
        projected on the bond `cur` by the MPS tensor A."""
        s = len(self.orbs)
        L = self.L
        I_site = site_op((), ())
        g = _Grow(A, self.sectors, cur, left=True)
        outside = _elementary(range(s + 1, L))
        N1, N2, C = {}, {}, {}
        for x, X in self.N1.items():
            N1[x] = g.build(1, X.dN, 1, [(1.0, I_site, X, 1)])
        for (o, d) in _elementary([s]):
            N1[(o, d)] = g.build(1, 1 if d == CREATE else -1, 1, [(1.0, site_op((d,), ()), None, 1)])
        for (pair, lab), X in self.N2.items():
            N2[(pair, lab)] = g.build(X.k, X.dN, 0, [(1.0, I_site, X, X.k)])
        for x, X in self.N1.items():
            for y in _elementary([s]):
                for lab in labelings(2):
                    K = lab[0]
                    dN, _ = _ops_meta((x, y))
                    N2[((x, y), lab)] = g.build(K, dN, 0, [(1.0, site_op((y[1],), ()), X, K)])
        sel = _elementary([s])
        for a in range(2):
            for b_ in range(a, 2):
                pair = (sel[a], sel[b_])
                for lab in labelings(2):
                    if not valid_labels(pair, lab):
                        continue
                    Y = site_op((pair[0][1], pair[1][1]), lab)
                    if Y is None:
                        continue
                    dN, _ = _ops_meta(pair)
                    N2[(pair, lab)] = g.build(lab[0], dN, 0, [(1.0, Y, None, lab[0])])
        for (O, lam) in _outside_keys(outside, 1):
            kO = lab_rank(len(O), lam)
            dN, par = _ops_meta(O)
            contribs = self._recursion(O, lam, s)
            if contribs:
                C[(O, lam)] = g.build(kO, -dN, par, contribs)
        b = LeftBlock(self.S, self.L)
        b.N1, b.N2, b.C = N1, N2, C
        b.orbs = self.orbs + [s]
        b.sectors = list(cur)
        return b

    def get(self, O, lam):
        if len(O) <= 1 and self.orbs:
            return self.C.get((O, lam))
        return self.direct(O, lam)

    def direct(self, O, lam, with_scalar=True):
        """C(O, lam) from the normal operators (|O| >= 2) or a number."""
        key = (O, lam, with_scalar)
        if key in self._direct_cache:
            return self._direct_cache[key]
        n = len(O)
        dN, par = _ops_meta(O)
        kO = lab_rank(n, lam)
        acc = None
        if n % 2 == 0 and with_scalar and kO == 0 and O in self.S:
            c = string_coef(lnest(n, lam), self.S[O])
            if c != 0.0:
                acc = _identity(self.sectors, c)
        if self.orbs and n >= 2:
            ops = _elementary(self.orbs)
            if n % 2 == 0 and n <= 2:                # two block factors
                for a in range(len(ops)):
                    for b in range(a, len(ops)):
                        pair = (ops[a], ops[b])
                        S = pair + O
                        if S not in self.S:
                            continue
                        for mu in labelings(2):
                            if not valid_labels(pair, mu) or mu[0] != kO:
                                continue
                            c = string_coef(("n", lnest(2, mu), lnest(n, lam), 0), self.S[S])
                            if c == 0.0:
                                continue
                            if acc is None:
                                acc = BOp(kO, -dN, 0, {})
                            acc.scaled_add(self.N2[(pair, mu)], c)
            elif n % 2 == 1 and kO == 1:             # one block factor
                for x in ops:
                    S = (x,) + O
                    if S not in self.S:
                        continue
                    c = string_coef(("n", E, lnest(n, lam), 0), self.S[S])
                    if c == 0.0:
                        continue
                    if acc is None:
                        acc = BOp(1, -dN, 1, {})
                    acc.scaled_add(self.N1[x], c)
        self._direct_cache[key] = acc
        return acc

    def _recursion(self, O1, lam1, s):
        k1 = lab_rank(len(O1), lam1)
        contribs = []
        for Y in [()] + site_strings(4 - len(O1)):
            nY = len(Y)
            Yops = tuple((s, d) for d in Y)
            O = Yops + O1
            for nu in labelings(nY):
                if nY and not valid_labels(Yops, nu):
                    continue
                Yop = site_op(Y, nu)
                if Yop is None:
                    continue
                kY = lab_rank(nY, nu)
                for lam in labelings(len(O)):
                    if not valid_labels(O, lam):
                        continue
                    kX = lab_rank(len(O), lam)
                    if not triangle(kX, kY, k1):
                        continue
                    W = overlap(("n", ("n", ("x", kX), lnest(nY, nu), k1), lnest(len(O1), lam1), 0),
                                ("n", ("x", kX), lnest(len(O), lam), 0))
                    if abs(W) < 1e-14:
                        continue
                    X = self.get(O, lam)
                    if X is None or X.k != kX:
                        continue
                    contribs.append((W, Yop, X, k1))
        return contribs


# ---------------------------------------------------------------------------
# the operator-table at the middle bond

def _split4(S, nL, p, q):
    A = tuple(x for x in S if x[0] < nL)
    B = tuple(x for x in S if x[0] == p)
    C = tuple(x for x in S if x[0] == q)
    D = tuple(x for x in S if x[0] > q)
    return A, B, C, D


def build_problem(cfg, h=None, eri=None):
    """(OperatorTable, env, left sectors, right sectors) of the ab initio
    Hamiltonian of cfg at its middle bond (left block cfg.n_left orbitals,
    sites p = n_left and q = n_left + 1, right block the rest), blocks from
    the seeded MPS.  Integrals default to ``synth.integrals``."""
    if h is None:
        h, eri = synth.integrals(cfg.L, cfg.seed)
    strings = hamiltonian_strings(h, eri)
    Lb = LeftBlock.seeded(strings, cfg, cfg.n_left)
    Rb = RightBlock.seeded(strings, cfg, cfg.n_right)
    return problem_from_blocks(strings, Lb, Rb)


def problem_from_blocks(strings, Lb, Rb):
    """(OperatorTable, env, left sectors, right sectors) at the two-site bond
    between a left block (orbitals 0 .. nL-1) and a right block (orbitals
    nL+2 .. L-1); sites p = nL, q = nL + 1."""
    nL = len(Lb.orbs)
    p, q = nL, nL + 1
    lsec, rsec = Lb.sectors, Rb.sectors
    table = model.OperatorTable(synth.SPATIAL_ORBITAL)
    env = {}
    lid, rid = {}, {}

    def op_id(side, key, bop):
        ids = lid if side == "L" else rid
        if key in ids:
            return ids[key]
        if bop is None:                              # identity
            oid = table.add_op(side, model.BlockOp("I", 0, 0, 0, model.IDENTITY))
        else:
            oid = table.add_op(side, model.BlockOp(str(key), bop.k, bop.dN, bop.parity, model.MPS_RENORM))
            sec = lsec if side == "L" else rsec
            blocks = {}
            for (qo, qi) in envmod.allowed_blocks(table.left_ops[oid] if side == "L" else table.right_ops[oid],
                                                  sec):
                M = bop.blocks.get((qo, qi))
                blocks[(qo, qi)] = M if M is not None else np.zeros((sec[qo][2], sec[qi][2]))
            env[(side, oid)] = blocks
        ids[key] = oid
        return oid

    IL = op_id("L", "I", None)
    IR = op_id("R", "I", None)
    # the block Hamiltonians first (left / right operator 1)
    if ((), ()) in Lb.C:
        op_id("L", ("C", (), ()), Lb.C[((), ())])
    if ((), ()) in Rb.C:
        op_id("R", ("C", (), ()), Rb.C[((), ())])

    def site_pairs(Bops, Cops):
        """Coupled site operators (labels, SiteOp) of the parts on sites p and q."""
        nB, nC = len(Bops), len(Cops)
        for beta in labelings(nB):
            if nB and not valid_labels(Bops, beta):
                continue
            Bs = site_op(tuple(d for _, d in Bops), beta)
            if Bs is None:
                continue
            for gamma in labelings(nC):
                if nC and not valid_labels(Cops, gamma):
                    continue
                Cs = site_op(tuple(d for _, d in Cops), gamma)
                if Cs is None:
                    continue
                yield beta, Bs, gamma, Cs

    # family (ii): left normal x sites x right complementary (the right
    # block Hamiltonian is the key O = ())
    rows = []
    right_keys = list(Rb.C.keys())
    # |O_R| = 3 combinations with at most one left factor
    outside_R = _elementary(list(range(nL)) + [p, q])
    for a in range(len(outside_R)):
        for b in range(a, len(outside_R)):
            for c in range(b, len(outside_R)):
                O = (outside_R[a], outside_R[b], outside_R[c])
                if sum(1 for x in O if x[0] < nL) > 1:
                    continue
                for lam in labelings(3):
                    if valid_labels(O, lam):
                        right_keys.append((O, lam))
    for (O, lam) in right_keys:
        X = Rb.get(O, lam)
        if X is None:
            continue
        n = len(O)
        kX = lab_rank(n, lam)
        if n == 2:                                   # remove the one-body part of strings outside R
            if kX == 0 and O in strings:
                c = string_coef(lnest(2, lam), strings[O])
                if c != 0.0:
                    X2 = BOp(X.k, X.dN, X.parity, dict(X.blocks))
                    X2.scaled_add(_identity(rsec), -c)
                    X = X2
        A, B, C, _ = _split4(O, nL, p, q)
        nA = len(A)
        src = ("n", lnest(n, lam), ("x", kX), 0)
        for alpha in labelings(nA):
            if nA and not valid_labels(A, alpha):
                continue
            kA = lab_rank(nA, alpha)
            if nA == 0:
                Aop_key, Aop = "I", None
            elif nA == 1:
                Aop_key, Aop = ("N1", A[0]), Lb.N1[A[0]]
            else:
                Aop_key, Aop = ("N2", A, alpha), Lb.N2.get((A, alpha))
                if Aop is None:
                    continue
            for beta, Bs, gamma, Cs in site_pairs(B, C):
                kB, kC = Bs.k, Cs.k
                for k in range(0, 9):
                    if not (triangle(kA, kB, k) and triangle(kC, kX, k)):
                        continue
                    dst = ("n", ("n", lnest(nA, alpha), lnest(len(B), beta), k),
                           ("n", lnest(len(C), gamma), ("x", kX), k), 0)
                    W = overlap(src, dst)
                    if abs(W) < 1e-14:
                        continue
                    rows.append((W, ("L", Aop_key, Aop), Bs, Cs, ("R", ("C", O, lam), X), k))
    # family (i): left complementary x sites x right normal
    left_keys = []
    sites_ops = _elementary([p, q])
    right_el = _elementary(list(range(q + 1, Lb.L)))
    for o in sites_ops + right_el:
        left_keys.append(((o,), ()))
    outside_L = sites_ops + right_el
    for a in range(len(sites_ops)):                  # |O_L| = 2: two site factors or one site + one right
        for b in range(a, len(outside_L)):
            O = (sites_ops[a], outside_L[b])
            for lam in labelings(2):
                if valid_labels(O, lam):
                    left_keys.append((O, lam))
    for a in range(len(sites_ops)):                  # |O_L| = 3: three site factors
        for b in range(a, len(sites_ops)):
            for c in range(b, len(sites_ops)):
                O = (sites_ops[a], sites_ops[b], sites_ops[c])
                for lam in labelings(3):
                    if valid_labels(O, lam):
                        left_keys.append((O, lam))
    for (O, lam) in left_keys:
        n = len(O)
        if n == 1:
            X = Lb.C.get((O, lam))
            if X is None:
                continue
            if O[0][0] > q:                          # remove the one-body part (it is in R's C(a_i))
                X2 = BOp(X.k, X.dN, X.parity, dict(X.blocks))
                for x in _elementary(Lb.orbs):
                    S = (x,) + O
                    if S in strings:
                        c = string_coef(("n", E, E, 0), strings[S]) if len(S) == 2 else 0.0
                        if c != 0.0:
                            X2.scaled_add(Lb.N1[x], -c)
                X = X2
        else:
            X = Lb.direct(O, lam, with_scalar=False)
            if X is None:
                continue
        kX = lab_rank(n, lam)
        _, B, C, D = _split4(O, nL, p, q)
        nD = len(D)
        src = ("n", ("x", kX), lnest(n, lam), 0)
        if nD == 0:
            Dop_key, Dop = "I", None
        else:
            Dop_key, Dop = ("N1", D[0]), Rb.N1[D[0]]
        kD = 1 if nD else 0
        for beta, Bs, gamma, Cs in site_pairs(B, C):
            kB, kC = Bs.k, Cs.k
            for k in range(0, 9):
                if not (triangle(kX, kB, k) and triangle(kC, kD, k)):
                    continue
                dst = ("n", ("n", ("x", kX), lnest(len(B), beta), k),
                       ("n", lnest(len(C), gamma), lnest(nD, ()), k), 0)
                W = overlap(src, dst)
                if abs(W) < 1e-14:
                    continue
                rows.append((W, ("L", ("C", O, lam), X), Bs, Cs, ("R", Dop_key, Dop), k))
    # H_L
    if ((), ()) in Lb.C:
        rows.append((1.0, ("L", ("C", (), ()), Lb.C[((), ())]), site_op((), ()), site_op((), ()),
                     ("R", "I", None), 0))
    # strings on the two sites only
    for S, F in strings.items():
        A, B, C, D = _split4(S, nL, p, q)
        if A or D:
            continue
        for beta, Bs, gamma, Cs in site_pairs(B, C):
            for k in range(0, 9):
                if not (triangle(0, Bs.k, k) and triangle(Cs.k, 0, k)):
                    continue
                t = ("n", ("n", ZERO, lnest(len(B), beta), k), ("n", lnest(len(C), gamma), ZERO, k), 0)
                W = string_coef(t, F)
                if abs(W) < 1e-14:
                    continue
                rows.append((W, ("L", "I", None), Bs, Cs, ("R", "I", None), k))
    for (W, (_, akey, aop), Bs, Cs, (_, dkey, dop), k) in rows:
        A = op_id("L", akey, aop)
        D = op_id("R", dkey, dop)
        table.terms.append(model.Term(W, A, Bs, Cs, D, k))
    return table, env, lsec, rsec
