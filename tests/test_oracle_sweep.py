"""Pins of the oracle's two-site sweep (Sec. II) on the ab initio Hamiltonian.

* With bonds that keep every multiplet, every step's Davidson energy is the
  full-CI ground-state energy (the two-site space is then the whole
  N-electron spin-0 space).
* With truncated bonds the energies are variational (never below full CI)
  and the discarded weights are non-negative.
* The SVD isometries: kept columns are orthonormal, the kept sectors hold at
  most D multiplets, and with D large enough nothing is discarded and the
  bond matrices are reproduced.
"""
import numpy as np

import synth
from oracle import fci, sectors, sweep


def test_exact_sweep_equals_full_ci_at_every_step():
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    E, w = sweep.sweep(cfg, 400, 2)
    h, eri = synth.integrals(6, 1002)
    e0 = fci.spin_levels(h, eri, 6, 0)[0]
    assert len(E) == 2 * (cfg.L - 1)
    assert np.abs(E - e0).max() < 1e-9
    assert np.all(np.abs(w) < 1e-20)


def test_truncated_sweep_is_variational():
    cfg = synth.Config("sw7", synth.SPATIAL_ORBITAL, 7, 6, 0, 6, 1002)
    E, w = sweep.sweep(cfg, 6, 2)
    h, eri = synth.integrals(7, 1002)
    e0 = fci.spin_levels(h, eri, 6, 0)[0]
    assert np.all(E >= e0 - 1e-10)
    assert np.all(w >= -1e-15) and w.max() > 0
    # the turn solves the same window twice
    assert abs(E[cfg.L - 2] - E[cfg.L - 1]) < 1e-9


def test_isometry_orthonormal_and_truncated():
    cfg = synth.Config("iso", synth.SPATIAL_ORBITAL, 8, 8, 0, 30, 3)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, 0)
    psi = synth.gaussian_psi(n, 4)
    for side in ("L", "R"):
        for D in (5, 10 ** 6):
            sec, A, w = sweep.isometry(psi, blocks, left, right, cfg.site_kind, cfg.N, D, side)
            assert sum(d for (_, _, d) in sec) <= D
            for qo, (rows, Q) in A.items():
                assert np.allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)
            if D > n:
                assert abs(w) < 1e-12
            else:
                assert w > 0
    # nothing discarded: U U^T reproduces every bond matrix
    mats = sweep._bond_matrices(psi, blocks, left, right, cfg.site_kind, cfg.N)
    sec, A, w = sweep.isometry(psi, blocks, left, right, cfg.site_kind, cfg.N, 10 ** 6, "L")
    keys = sorted(mats)
    for qo, (Nb, j, d) in enumerate(sec):
        rows, U = A[qo]
        M = mats[(Nb, j)][2]
        assert np.allclose(U @ (U.T @ M), M, atol=1e-12)
