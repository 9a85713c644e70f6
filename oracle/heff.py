"""Sector-task-table, sector-value table and H.psi (Eqs. 2-3, Sec. II.C).

Oracle module (test infrastructure only).  For every operator-table row i
and every input block e the reachable output blocks f are enumerated; each
(i, e, f) is one row of the sector-task-table of Eq. 3 with pointers to the
left operator block A_i{p^A}, the input block E{p^E}, the right operator
block D_i{p^D} and the output block F{p^F}.  The site operators B_i, C_i
act on one-dimensional sectors, so their reduced elements, alpha_i and the
three Clebsch-Gordan-layer factors C~ (Eq. a) fold into one scalar per task
(the sector-value table):

    v = alpha_i * <s1'||B||s1> <s2'||C||s2> * C~_l * C~_r * C~_h * sign,
    C~_l = C~(S_a, s1, jL1; kA, kB, k; S_a', s1', jL1')     W9j^(l)
    C~_r = C~(s2, S_b, j2R; kC, kD, k; s2', S_b', j2R')     W9j^(r)
    C~_h = C~(jL1, j2R, S; k, k, 0; jL1', j2R', S)          W9j^(h)
    sign = (-1)^{pB N_a + pC (N_a + n1) + pD (N_a + n1 + n2)}

(fermionic order: left block, site 1, site 2, right block).  The task then
computes F{f} += v * A{a'<-a} . E{e} . D{b'<-b}^T.

Tasks are selected by integer rules only (particle number, triangle
conditions, structural non-zeros of the site operators); a coefficient that
vanishes accidentally keeps its task with v = 0.  Tasks are ordered by
(f, i, e), which is also the summation order of ``apply_heff``.

Parity: ``apply_heff`` is pinned against the m-resolved expansion and the
explicit full-space projection in ``expand`` and against exact
diagonalisation (Heisenberg), plus Hermiticity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import synth
from .model import IDENTITY, OperatorTable
from .sectors import Block, block_index, block_view, couple
from .su2 import ctilde, triangle


@dataclass(frozen=True)
class Task:
    f: int
    term: int
    e: int
    A: tuple      # (a_out, a_in) or None for the identity
    D: tuple      # (b_out, b_in) or None for the identity
    v: float


def _out_sectors(op, sectors, a):
    """Sectors reachable from sector a by a block operator (or identity)."""
    if op.kind == IDENTITY:
        return [a]
    Na, Sa, _ = sectors[a]
    res = []
    for ap, (Np, Sp, _) in enumerate(sectors):
        if Np == Na + op.dN and triangle(Sa, op.k, Sp):
            res.append(ap)
    return res


def build_tasks(table: OperatorTable, left, right, blocks, twoS_target, only_f=None):
    """Sector-task-table; ``only_f`` (a set of output block indices) keeps
    only the tasks writing into those blocks (sampled checks of large
    problems)."""
    sk = table.site_kind
    sites = synth.site_states(sk)
    bidx = block_index(blocks)
    S = twoS_target
    tasks = []
    for ti, term in enumerate(table.terms):
        Aop = table.left_ops[term.A]
        Dop = table.right_ops[term.D]
        Bm, Cm = term.B.mat(), term.C.mat()
        k = term.k
        for e, E in enumerate(blocks):
            Na, Sa, _ = left[E.a]
            n1, t1 = sites[E.s1]
            n2, t2 = sites[E.s2]
            Nb, Sb, _ = right[E.b]
            sexp = term.B.parity * Na + term.C.parity * (Na + n1) + Dop.parity * (Na + n1 + n2)
            sign = -1.0 if sexp % 2 else 1.0
            for ap in _out_sectors(Aop, left, E.a):
                Sap = left[ap][1]
                for s1p in range(len(sites)):
                    bval = Bm[s1p, E.s1]
                    if bval == 0.0:
                        continue
                    t1p = sites[s1p][1]
                    for s2p in range(len(sites)):
                        cval = Cm[s2p, E.s2]
                        if cval == 0.0:
                            continue
                        t2p = sites[s2p][1]
                        for bp in _out_sectors(Dop, right, E.b):
                            Sbp = right[bp][1]
                            for jL1p in couple(Sap, t1p):
                                if not triangle(E.jL1, k, jL1p):
                                    continue
                                for j2Rp in couple(t2p, Sbp):
                                    if not triangle(E.j2R, k, j2Rp) or not triangle(jL1p, j2Rp, S):
                                        continue
                                    f = bidx.get((ap, s1p, s2p, bp, jL1p, j2Rp))
                                    if f is None or (only_f is not None and f not in only_f):
                                        continue
                                    cl = ctilde(Sa, t1, E.jL1, Aop.k, term.B.k, k, Sap, t1p, jL1p)
                                    cr = ctilde(t2, Sb, E.j2R, term.C.k, Dop.k, k, t2p, Sbp, j2Rp)
                                    ch = ctilde(E.jL1, E.j2R, S, k, k, 0, jL1p, j2Rp, S)
                                    v = term.alpha * bval * cval * cl * cr * ch * sign
                                    tasks.append(Task(f, ti, e,
                                                      None if Aop.kind == IDENTITY else (ap, E.a),
                                                      None if Dop.kind == IDENTITY else (bp, E.b),
                                                      v))
    tasks.sort(key=lambda t: (t.f, t.term, t.e))
    return tasks


def apply_heff(table, env, tasks, blocks, psi_len, psi):
    """F = H_eff psi as the sum of Eq. 2 over the sector-task-table, FP64.

    ``env`` maps (side, op id) -> {(out sector, in sector): matrix}.  With a
    task list restricted to some output blocks, only those blocks of F are
    computed (the rest stays zero).
    """
    F = np.zeros(psi_len)
    for t in tasks:
        E = block_view(psi, blocks[t.e])
        term = table.terms[t.term]
        X = E
        if t.D is not None:
            X = X @ env[("R", term.D)][t.D].T
        if t.A is not None:
            X = env[("L", term.A)][t.A] @ X
        Fb = block_view(F, blocks[t.f])
        Fb += t.v * X
    return F


def diag_heff(table, env, tasks, blocks, psi_len):
    """Diagonal of H_eff: tasks with e == f contribute v * A_xx * D_yy."""
    d = np.zeros(psi_len)
    for t in tasks:
        if t.e != t.f:
            continue
        B = blocks[t.f]
        term = table.terms[t.term]
        a = np.ones(B.rows) if t.A is None else np.diag(env[("L", term.A)][t.A]).copy()
        b = np.ones(B.cols) if t.D is None else np.diag(env[("R", term.D)][t.D]).copy()
        block_view(d, B)[...] += t.v * np.outer(a, b)
    return d


def flops(tasks, blocks):
    """SU(2) flops of one H.psi for the association executed (E D^T first,
    then A times it): 2 m k1 k2... counted per task, identities skipped."""
    tot = 0
    for t in tasks:
        E, Fb = blocks[t.e], blocks[t.f]
        m, k1, k2, n = Fb.rows, E.rows, E.cols, Fb.cols
        if t.D is not None:
            tot += 2 * k1 * k2 * n
        if t.A is not None:
            tot += 2 * m * k1 * n
    return tot
