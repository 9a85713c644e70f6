"""Reduced site operators and the operator-table of Eq. 2.

Oracle module (test infrastructure only).  Every operator is stored as a
*reduced* matrix in the Clebsch-Gordan form of the Wigner-Eckart theorem,
<j' m'|T^k_q|j m> = <j m; k q|j' m'> <j'||T^k||j>  (Sec. II.B: reduced
operators of dimension three for a spin-1/2 fermion site).  Spins and ranks
are twos integers.

H.psi of Eq. 2 is a sum over operator-table rows i of
    alpha_i [[A_i^{kA} x B_i^{kB}]^{k_i} x [C_i^{kC} x D_i^{kD}]^{k_i}]^0,
A_i on the left block, B_i on site 1, C_i on site 2, D_i on the right
block.  The coupling order (L s1)(s2 R) is the one whose factors are the
W9j^(l), W9j^(r) and W9j^(h) tables of Sec. II.C.

Parity: pinned by ``expand`` (m-resolved expansion, Hermiticity) and, for the
Heisenberg chain, by exact diagonalisation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

import synth


@dataclass(frozen=True)
class SiteOp:
    name: str
    k: int          # rank, twos
    dN: int
    parity: int     # fermion parity of the operator (0 even, 1 odd)
    red: tuple      # reduced matrix red[out_state][in_state] as nested tuples

    def mat(self) -> np.ndarray:
        return np.array(self.red, dtype=np.float64)


def site_twoS(site_kind):
    return [s for (_, s) in synth.site_states(site_kind)]


def site_N(site_kind):
    return [n for (n, _) in synth.site_states(site_kind)]


def adjoint_reduced(red: np.ndarray, k: int, twoS_out, twoS_in) -> np.ndarray:
    """Reduced matrix of the adjoint tensor T^dag_q = (-1)^{k-q} (T_{-q})^+.

    With the Clebsch-Gordan form of Wigner-Eckart,
    <a||T^dag||b> = (-1)^{(S_b + k - S_a)} sqrt((2S_b+1)/(2S_a+1)) <b||T||a>.
    ``red`` is [out][in] for T with out spins ``twoS_out`` and in spins
    ``twoS_in``; the result is [out][in] for T^dag, i.e. out spins twoS_in.
    """
    res = np.zeros((red.shape[1], red.shape[0]))
    for a in range(red.shape[1]):          # T^dag out = T in
        for b in range(red.shape[0]):      # T^dag in  = T out
            if red[b, a] == 0.0:
                continue
            e = twoS_out[b] + k - twoS_in[a]
            assert e % 2 == 0
            sign = -1.0 if (e // 2) % 2 else 1.0
            res[a, b] = sign * math.sqrt((twoS_out[b] + 1) / (twoS_in[a] + 1)) * red[b, a]
    return res


def _tup(m):
    return tuple(tuple(float(x) for x in row) for row in m)


def site_ops(site_kind):
    """Dictionary of the reduced site operators of a site kind.

    Orbital site states (|0>, |sigma>, |2>) = ((N=0,S=0), (1,1/2), (2,0)).
    a^+ (k=1/2): <sigma||a^+||0> = 1, <2||a^+||sigma> = -sqrt(2)
    (from c^+_up c^+_dn|0> = |2>).  a~ is the adjoint tensor of a^+.
    S (k=1): <sigma||S||sigma> = sqrt(3/4).  pair = [a^+ x a^+]^0 = sqrt(2)
    c^+_up c^+_dn.  Spin-1/2 site: a single multiplet with identity and S.
    """
    tw = site_twoS(site_kind)
    ops = {}
    if site_kind == synth.SPIN_HALF:
        ops["I"] = SiteOp("I", 0, 0, 0, ((1.0,),))
        ops["S"] = SiteOp("S", 2, 0, 0, ((math.sqrt(0.75),),))
        return ops
    I = np.eye(3)
    n = np.diag([0.0, 1.0, 2.0])
    dbl = np.diag([0.0, 0.0, 1.0])
    cdag = np.zeros((3, 3)); cdag[1, 0] = 1.0; cdag[2, 1] = -math.sqrt(2.0)
    S = np.zeros((3, 3)); S[1, 1] = math.sqrt(0.75)
    pair = np.zeros((3, 3)); pair[2, 0] = math.sqrt(2.0)
    ops["I"] = SiteOp("I", 0, 0, 0, _tup(I))
    ops["n"] = SiteOp("n", 0, 0, 0, _tup(n))
    ops["dbl"] = SiteOp("dbl", 0, 0, 0, _tup(dbl))
    ops["cdag"] = SiteOp("cdag", 1, +1, 1, _tup(cdag))
    ops["c"] = SiteOp("c", 1, -1, 1, _tup(adjoint_reduced(cdag, 1, tw, tw)))
    ops["S"] = SiteOp("S", 2, 0, 0, _tup(S))
    ops["pair"] = SiteOp("pair", 0, +2, 0, _tup(pair))
    ops["pairdag"] = SiteOp("pairdag", 0, -2, 0, _tup(adjoint_reduced(pair, 0, tw, tw)))
    return ops


def site_adjoint(op: SiteOp, site_kind) -> SiteOp:
    tw = site_twoS(site_kind)
    return SiteOp(op.name + "^+", op.k, -op.dN, op.parity,
                  _tup(adjoint_reduced(op.mat(), op.k, tw, tw)))


# ---------------------------------------------------------------------------
# block operators: descriptors only (values live in ``env``)

IDENTITY, HAM, RANDOM, ADJOINT, MPS_RENORM, SPINTOT, NUMTOT = range(7)


@dataclass
class BlockOp:
    """One block operator of a side ('L' or 'R').

    kind: IDENTITY, HAM (scalar Hamiltonian of the block), RANDOM (seeded
    synthetic entries), ADJOINT (adjoint tensor of op ``base``), MPS_RENORM
    (renormalised from an MPS; Heisenberg only), SPINTOT (total spin of the
    block, reduced element sqrt(S(S+1)) on each sector), NUMTOT (particle
    number of the block, N on each sector).
    """
    name: str
    k: int
    dN: int
    parity: int
    kind: int
    base: int = -1


@dataclass
class Term:
    """Operator-table row of Eq. 2: alpha, A (left op id), B, C (site ops),
    D (right op id), coupling rank k (twos) of [A x B] and [C x D]."""
    alpha: float
    A: int
    B: SiteOp
    C: SiteOp
    D: int
    k: int


@dataclass
class OperatorTable:
    site_kind: int
    left_ops: list = field(default_factory=list)
    right_ops: list = field(default_factory=list)
    terms: list = field(default_factory=list)

    def add_op(self, side, op: BlockOp) -> int:
        lst = self.left_ops if side == "L" else self.right_ops
        lst.append(op)
        return len(lst) - 1

    def add_random_pair(self, side, name, k, dN, parity):
        """A seeded random operator and its adjoint tensor; returns both ids."""
        i = self.add_op(side, BlockOp(name, k, dN, parity, RANDOM))
        j = self.add_op(side, BlockOp(name + "^+", k, -dN, parity, ADJOINT, i))
        return i, j

    def adjoint_id(self, side, oid):
        lst = self.left_ops if side == "L" else self.right_ops
        op = lst[oid]
        if op.kind in (IDENTITY, HAM):
            return oid
        if op.kind == ADJOINT:
            return op.base
        for j, o in enumerate(lst):
            if o.kind == ADJOINT and o.base == oid:
                return j
        raise KeyError(oid)

    def add_term_hc(self, alpha, A, B, C, D, k):
        """Append a term and its Hermitian conjugate.

        (alpha O)^+ with O = [[A x B]^k x [C x D]^k]^0 equals
        alpha * (-1)^{pX pY + pA pB + pC pD} [[A^+ x B^+]^k x [C^+ x D^+]^k]^0
        (pX = pA + pB, pY = pC + pD; fermionic reordering signs).
        """
        self.terms.append(Term(alpha, A, B, C, D, k))
        pA = self.left_ops[A].parity
        pD = self.right_ops[D].parity
        pB, pC = B.parity, C.parity
        e = (pA + pB) * (pC + pD) + pA * pB + pC * pD
        sgn = -1.0 if e % 2 else 1.0
        self.terms.append(Term(alpha * sgn, self.adjoint_id("L", A),
                               site_adjoint(B, self.site_kind),
                               site_adjoint(C, self.site_kind),
                               self.adjoint_id("R", D), k))


def heisenberg_table(J: float = 1.0) -> OperatorTable:
    """Two-site terms of H = J sum_i S_i.S_{i+1} at a bond (Sec. II.A form).

    S_a.S_b = -sqrt(3) [S_a x S_b]^0.  Block operators: identity, H_block and
    S_edge (the spin of the block site next to the two-site window).
    Rows: H_L, S_L.s1, s1.s2, s2.S_R, H_R.
    """
    t = OperatorTable(synth.SPIN_HALF)
    ops = site_ops(synth.SPIN_HALF)
    I, S = ops["I"], ops["S"]
    for side in ("L", "R"):
        t.add_op(side, BlockOp("I", 0, 0, 0, IDENTITY))
        t.add_op(side, BlockOp("H", 0, 0, 0, MPS_RENORM))
        t.add_op(side, BlockOp("S", 2, 0, 0, MPS_RENORM))
    c = -math.sqrt(3.0) * J
    t.terms.append(Term(1.0, 1, I, I, 0, 0))      # H_L
    t.terms.append(Term(c, 2, S, I, 0, 0))        # S_L . s1
    t.terms.append(Term(c, 0, S, S, 0, 2))        # s1 . s2
    t.terms.append(Term(c, 0, I, S, 2, 0))        # s2 . S_R
    t.terms.append(Term(1.0, 0, I, I, 1, 0))      # H_R
    return t


def qc_skeleton_table(n_left: int, n_right: int) -> OperatorTable:
    """Operator-table with the term structure of the ab initio Hamiltonian in
    the normal/complementary partition (left block: normal operators with up
    to two orbital indices; right block: complementary operators), synthetic
    entries.  The families and their order are the canonical order shared
    with the library:

    F1  H_L x 1 x 1 x 1, 1 x 1 x 1 x H_R
    F2  site one-body and on-site terms n, n_up n_dn on sites 1 and 2
    F3  site1-site2: hopping (+h.c.), S.S, n n, pair hopping (+h.c.)
    F4  a^+_i x 1 x 1 x Sbar_i^R (+h.c.), i in L
    F5  [a^+_i x a~_p]^k x [1 x Q_ip^{R,k}] (+h.c.), k=0,1;
        [a^+_i x 1]^{1/2} x [a~_q x Q_iq^{R,k}]^{1/2} (+h.c.), k=0,1
    F6  A_ij^k x 1 x 1 x P_ij^{R,k} (+h.c.), B_ij^k x 1 x 1 x Q_ij^{R,k}
        (+h.c.), i<=j in L, k=0,1 (k=1 only for i<j for A)
    F7  S_l^L x 1 x 1 x a~_l^R (+h.c.), l in R
    F8  1 x a^+_p x 1 x Sbar_p^R (+h.c.), 1 x 1 x a^+_q x Sbar_q^R (+h.c.)
    F9  [S_p^L x a~_p]^0 x 1 x 1 (+h.c.), [S_q^L x 1]^{1/2} x [a~_q x 1] (+h.c.)

    Coefficients alpha: 1 (F1), 1/2 (F2, F3, F8, F9), 1/sqrt(n_left) (F4,
    F5), 1/n_left (F6), 1/sqrt(n_right) (F7).
    """
    sk = synth.SPATIAL_ORBITAL
    t = OperatorTable(sk)
    so = site_ops(sk)
    I, n, dbl, cdag, c, S, pair, pairdag = (so[x] for x in
                                            ("I", "n", "dbl", "cdag", "c", "S", "pair", "pairdag"))
    IL = t.add_op("L", BlockOp("I", 0, 0, 0, IDENTITY))
    HL = t.add_op("L", BlockOp("H", 0, 0, 0, HAM))
    IR = t.add_op("R", BlockOp("I", 0, 0, 0, IDENTITY))
    HR = t.add_op("R", BlockOp("H", 0, 0, 0, HAM))
    wL1 = 1.0 / math.sqrt(n_left)
    wL2 = 1.0 / n_left
    wR1 = 1.0 / math.sqrt(n_right)
    # F1
    t.terms.append(Term(1.0, HL, I, I, IR, 0))
    t.terms.append(Term(1.0, IL, I, I, HR, 0))
    # F2
    for op in (n, dbl):
        t.terms.append(Term(0.5, IL, op, I, IR, 0))
    for op in (n, dbl):
        t.terms.append(Term(0.5, IL, I, op, IR, 0))
    # F3
    t.add_term_hc(0.5, IL, cdag, c, IR, 1)
    t.terms.append(Term(0.5, IL, S, S, IR, 2))
    t.terms.append(Term(0.5, IL, n, n, IR, 0))
    t.add_term_hc(0.5, IL, pair, pairdag, IR, 0)
    # F4
    for i in range(n_left):
        a, _ = t.add_random_pair("L", f"a+_{i}", 1, +1, 1)
        sb, _ = t.add_random_pair("R", f"Sbar_{i}", 1, -1, 1)
        t.add_term_hc(wL1, a, I, I, sb, 1)
    # F5
    for i in range(n_left):
        a = [o for o, op in enumerate(t.left_ops) if op.name == f"a+_{i}"][0]
        for k in (0, 2):
            q, _ = t.add_random_pair("R", f"Q_{i}p^{k}", k, 0, 0)
            t.add_term_hc(wL1, a, c, I, q, k)
        for k in (0, 2):
            q, _ = t.add_random_pair("R", f"Q_{i}q^{k}", k, 0, 0)
            t.add_term_hc(wL1, a, I, c, q, 1)
    # F6
    for i in range(n_left):
        for j in range(i, n_left):
            for k in (0, 2):
                if k == 2 and i == j:
                    continue
                A, _ = t.add_random_pair("L", f"A_{i}{j}^{k}", k, +2, 0)
                P, _ = t.add_random_pair("R", f"P_{i}{j}^{k}", k, -2, 0)
                t.add_term_hc(wL2, A, I, I, P, k)
            for k in (0, 2):
                B, _ = t.add_random_pair("L", f"B_{i}{j}^{k}", k, 0, 0)
                Q, _ = t.add_random_pair("R", f"Q_{i}{j}^{k}", k, 0, 0)
                t.add_term_hc(wL2, B, I, I, Q, k)
    # F7
    for l in range(n_right):
        SL, _ = t.add_random_pair("L", f"S_{l}", 1, +1, 1)
        aR, _ = t.add_random_pair("R", f"a~_{l}", 1, -1, 1)
        t.add_term_hc(wR1, SL, I, I, aR, 1)
    # F8
    sp, _ = t.add_random_pair("R", "Sbar_p", 1, -1, 1)
    t.add_term_hc(0.5, IL, cdag, I, sp, 1)
    sq, _ = t.add_random_pair("R", "Sbar_q", 1, -1, 1)
    t.add_term_hc(0.5, IL, I, cdag, sq, 0)
    # F9
    Sp, _ = t.add_random_pair("L", "S_p", 1, +1, 1)
    t.add_term_hc(0.5, Sp, c, I, IR, 0)
    Sq, _ = t.add_random_pair("L", "S_q", 1, +1, 1)
    t.add_term_hc(0.5, Sq, I, c, IR, 1)
    return t


def casimir_table(site_kind, which):
    """Operator-table of S_tot^2 (which='S2') or N_tot (which='N') over the
    four subsystems, written with the block total-spin / number operators.

    S_tot^2 = sum_X S_X^2 + 2 sum_{X<Y} S_X.S_Y with S_X.S_Y = -sqrt(3)
    [S_X x S_Y]^0 and S_X^2 = sqrt(3)... written as -sqrt(3)[S_X x S_X]^0 on
    one subsystem, i.e. the scalar S(S+1).  Applied to a psi of total spin S
    it must return S(S+1) psi; N_tot must return N psi.  Both hold exactly
    for any sector dimensions because the two-site space is a sum of whole
    multiplets.
    """
    t = OperatorTable(site_kind)
    so = site_ops(site_kind)
    I = so["I"]
    for side in ("L", "R"):
        t.add_op(side, BlockOp("I", 0, 0, 0, IDENTITY))
        t.add_op(side, BlockOp("S", 2, 0, 0, SPINTOT))
        t.add_op(side, BlockOp("N", 0, 0, 0, NUMTOT))
    if which == "N":
        n_site = so["n"] if site_kind == synth.SPATIAL_ORBITAL else SiteOp("n", 0, 0, 0, ((1.0,),))
        t.terms.append(Term(1.0, 2, I, I, 0, 0))
        t.terms.append(Term(1.0, 0, n_site, I, 0, 0))
        t.terms.append(Term(1.0, 0, I, n_site, 0, 0))
        t.terms.append(Term(1.0, 0, I, I, 2, 0))
        return t
    S = so["S"]
    c = -math.sqrt(3.0)
    # squares: S_L^2 and S_R^2 as [S x S]^0 products of the block operator
    # with itself are not single operators here, so use the site-free forms
    # S_L.S_L = -sqrt(3) [[S_L x 1]^1 x [1 x 1]]... is not expressible as one
    # row; instead the squares enter through the reduced identity
    # S_X^2 = S_X(S_X+1) handled by NUMTOT-like diagonal rows below.
    t.add_op("L", BlockOp("S2", 0, 0, 0, SPINTOT))
    t.add_op("R", BlockOp("S2", 0, 0, 0, SPINTOT))
    s2site = SiteOp("S2", 0, 0, 0, tuple(tuple(float(0.75 if (i == j and S.red[i][i] != 0.0) else 0.0)
                                                     for j in range(len(S.red))) for i in range(len(S.red))))
    t.terms.append(Term(1.0, 3, I, I, 0, 0))          # S_L^2
    t.terms.append(Term(1.0, 0, s2site, I, 0, 0))     # s1^2
    t.terms.append(Term(1.0, 0, I, s2site, 0, 0))     # s2^2
    t.terms.append(Term(1.0, 0, I, I, 3, 0))          # S_R^2
    t.terms.append(Term(2 * c, 1, S, I, 0, 0))        # 2 S_L.s1   [[S_L x s1]^0 x 1]
    t.terms.append(Term(2 * c, 1, I, S, 0, 2))        # 2 S_L.s2   [[S_L x 1]^1 x [s2 x 1]^1]^0
    t.terms.append(Term(2 * c, 1, I, I, 1, 2))        # 2 S_L.S_R
    t.terms.append(Term(2 * c, 0, S, S, 0, 2))        # 2 s1.s2
    t.terms.append(Term(2 * c, 0, S, I, 1, 2))        # 2 s1.S_R
    t.terms.append(Term(2 * c, 0, I, S, 1, 0))        # 2 s2.S_R   [1 x [s2 x S_R]^0]
    return t
