"""Exact diagonalisation of the open spin-1/2 Heisenberg chain.

Oracle module (test infrastructure only).  Dense Hamiltonian in the sector
with fixed S_z = twoM/2, H = J sum_i S_i.S_{i+1}; eigenvalues by a dense
symmetric eigensolver.  Pins: two sites give -3/4 J (singlet); L=4 gives
the known closed form -(3/4 + sqrt(3)/2) J... checked in the tests.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np


def heisenberg_sector(L, twoM, J=1.0):
    n_up = (L + twoM) // 2
    states = []
    for ups in combinations(range(L), n_up):
        s = 0
        for u in ups:
            s |= 1 << u
        states.append(s)
    index = {s: i for i, s in enumerate(states)}
    H = np.zeros((len(states), len(states)))
    for i, s in enumerate(states):
        for b in range(L - 1):
            u1 = (s >> b) & 1
            u2 = (s >> (b + 1)) & 1
            H[i, i] += J * (0.25 if u1 == u2 else -0.25)
            if u1 != u2:
                t = s ^ (1 << b) ^ (1 << (b + 1))
                H[index[t], i] += 0.5 * J
    return H


def heisenberg_levels(L, twoM, J=1.0):
    return np.linalg.eigvalsh(heisenberg_sector(L, twoM, J))
