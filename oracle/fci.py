"""Full configuration interaction for small ab initio Hamiltonians (Eq. 1).

Oracle module (test infrastructure only).  The Hamiltonian
    H = sum_ij h_ij sum_s c+_is c_js + 1/2 sum_ijkl (ij|kl) sum_st c+_is c+_kt c_lt c_js
is built as a sparse matrix on the Fock space of L spatial orbitals
(spin-orbital 2i + s, s = 0 up, 1 down; Jordan-Wigner order by spin-orbital
index, so that an orbital's doubly occupied state is c+_up c+_dn |0>).  A
basis state is a bit pattern of occupied spin-orbitals; c+_p carries the
sign (-1)^(number of occupied spin-orbitals below p).

The spin-S multiplets of the N-electron space are the eigenvalues of the
S_z = S block that do not also occur in the S_z = S + 1 block (every
multiplet of spin S' > S has a member in both).

Parity: pinned by closed forms in the tests (one doubly occupied orbital:
2 h + (00|00); no two-body part: twice the sum of the lowest N/2 orbital
energies), Hermiticity and particle-number / spin conservation.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


def _sector_states(L, N, twoSz):
    n_up = (N + twoSz) // 2
    n_dn = (N - twoSz) // 2
    if n_up < 0 or n_dn < 0 or n_up > L or n_dn > L or (N + twoSz) % 2:
        return []
    states = []
    for ups in itertools.combinations(range(L), n_up):
        for dns in itertools.combinations(range(L), n_dn):
            s = 0
            for i in ups:
                s |= 1 << (2 * i)
            for i in dns:
                s |= 1 << (2 * i + 1)
            states.append(s)
    return sorted(states)


def _apply(ops, s):
    """Apply a product of (mode, create) operators, rightmost first, to the
    bit pattern s; returns (sign, new pattern) or None."""
    sign = 1
    for (p, create) in reversed(ops):
        occ = (s >> p) & 1
        if create == occ:
            return None
        below = bin(s & ((1 << p) - 1)).count("1")
        if below % 2:
            sign = -sign
        s ^= 1 << p
    return sign, s


def hamiltonian_sector(h, eri, N, twoSz):
    """Dense H on the (N, S_z) determinant space and its basis."""
    L = h.shape[0]
    states = _sector_states(L, N, twoSz)
    index = {s: i for i, s in enumerate(states)}
    n = len(states)
    rows, cols, vals = [], [], []
    terms = []
    for i in range(L):
        for j in range(L):
            if h[i, j] != 0.0:
                for s_ in (0, 1):
                    terms.append((h[i, j], [(2 * i + s_, 1), (2 * j + s_, 0)]))
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = eri[i, j, k, l]
                    if v == 0.0:
                        continue
                    for s_ in (0, 1):
                        for t_ in (0, 1):
                            terms.append((0.5 * v, [(2 * i + s_, 1), (2 * k + t_, 1), (2 * l + t_, 0),
                                                    (2 * j + s_, 0)]))
    for col, s in enumerate(states):
        for (c, ops) in terms:
            r = _apply(ops, s)
            if r is None:
                continue
            sign, t = r
            rows.append(index[t])
            cols.append(col)
            vals.append(sign * c)
    H = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).toarray()
    return H, states


def spin_levels(h, eri, N, twoS):
    """Sorted eigenvalues of the spin-S multiplets of the N-electron space."""
    H0, _ = hamiltonian_sector(h, eri, N, twoS)
    H1, st1 = hamiltonian_sector(h, eri, N, twoS + 2)
    e0 = list(np.linalg.eigvalsh(H0)) if H0.size else []
    e1 = list(np.linalg.eigvalsh(H1)) if H1.size else []
    e0.sort()
    for x in e1:
        j = int(np.argmin([abs(y - x) for y in e0]))
        assert abs(e0[j] - x) <= 1e-8 * max(1.0, abs(x)), (x, e0[j])
        e0.pop(j)
    return np.array(e0)
