"""Block-sparse two-site wavefunction (sector-table of Sec. II.A).

Oracle module (test infrastructure only).  A block of psi is labelled by
(a, s1, s2, b, jL1, j2R): left-block sector a, site states s1 and s2,
right-block sector b, and the intermediate spins of the couplings
(a x s1) -> jL1 and (s2 x b) -> j2R, with jL1 x j2R -> S_target (the
coupling order of the W9j^(l), W9j^(r), W9j^(h) factors, Sec. II.C).  Each
block is a dense d_a x d_b column-major FP64 matrix; blocks are stored one
after another in the canonical order of the nested loops below.

Parity: the block list is bit-exact against the library
(``tests/test_lib_host.py``) and pinned in ``tests/test_oracle_abinitio.py``:
sum_blocks d_a d_b equals an independent count of the spin-S multiplets of
(S_a x s1 x s2 x S_b) by characters (states with M = S minus M = S + 1) on
truncated bonds, and the Weyl-Paldus number of spin-S multiplets of N
electrons in L orbitals when the bonds keep every multiplet.
"""
from __future__ import annotations

from dataclasses import dataclass

import synth
from .su2 import triangle


@dataclass(frozen=True)
class Block:
    a: int
    s1: int
    s2: int
    b: int
    jL1: int
    j2R: int
    rows: int
    cols: int
    offset: int


def couple(x: int, y: int):
    return range(abs(x - y), x + y + 1, 2)


def build_blocks(left, right, site_kind, N_target, twoS_target):
    """All psi blocks and the total length.  ``left``/``right`` are lists of
    (N, 2S, d) bond sectors in the caller's order."""
    sites = synth.site_states(site_kind)
    blocks = []
    off = 0
    for a, (Na, Sa, da) in enumerate(left):
        for s1, (n1, t1) in enumerate(sites):
            for s2, (n2, t2) in enumerate(sites):
                for b, (Nb, Sb, db) in enumerate(right):
                    if Na + n1 + n2 + Nb != N_target:
                        continue
                    for jL1 in couple(Sa, t1):
                        for j2R in couple(t2, Sb):
                            if not triangle(jL1, j2R, twoS_target):
                                continue
                            blocks.append(Block(a, s1, s2, b, jL1, j2R, da, db, off))
                            off += da * db
    return blocks, off


def block_index(blocks):
    return {(B.a, B.s1, B.s2, B.b, B.jL1, B.j2R): i for i, B in enumerate(blocks)}


def block_view(vec, B: Block):
    """Column-major d_a x d_b view of block B inside a flat psi vector."""
    return vec[B.offset:B.offset + B.rows * B.cols].reshape(B.cols, B.rows).T
