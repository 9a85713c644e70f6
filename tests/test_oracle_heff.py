"""Pins of the oracle's sector-form H.psi (Eqs. 2-3, Sec. II.C).

* Casimir operators through the same machinery: S_tot^2 psi = S(S+1) psi and
  N_tot psi = N psi, for targets S = 0, 1/2, 1, 3/2 (exact; the two-site
  space is a sum of whole multiplets).
* The m-resolved (U(1)) expansion with Clebsch-Gordan coefficients, which
  uses no 6j/9j, on the ab initio skeleton with fermionic operators.
* Hermiticity of H_eff and the diagonal of H_eff.
* Heisenberg chains: explicit full-space projection P^T H P of the same
  seeded MPS, and exact diagonalisation (a full-basis MPS makes H_eff the
  whole singlet sector, so its lowest eigenvalue is the exact energy).
* A planted mistake (the transposed coupling order in C~) must be caught.
"""
import math

import numpy as np
import pytest

import synth
from oracle import davidson, ed, env, expand, heff, model, sectors, su2

LEFT = [(1, 1, 2), (2, 0, 1), (2, 2, 1), (3, 1, 1)]
RIGHT = [(1, 1, 1), (2, 0, 1), (2, 2, 1), (3, 1, 1)]
LEFT_W = [(1, 1, 2), (2, 0, 2), (2, 2, 1), (3, 1, 2), (3, 3, 1)]
RIGHT_W = [(1, 1, 1), (2, 0, 2), (2, 2, 2), (3, 1, 1)]


def _setup(table, left, right, sk, N, S, seed=7):
    blocks, n = sectors.build_blocks(left, right, sk, N, S)
    cfg = synth.Config("t", sk, 8, N, S, 8, seed)
    e = env.build_env(table, cfg, left, right)
    tasks = heff.build_tasks(table, left, right, blocks, S)
    return blocks, n, e, tasks


@pytest.mark.parametrize("N,S", [(6, 0), (6, 2), (5, 1), (7, 3)])
@pytest.mark.parametrize("which", ["S2", "N"])
def test_casimir(N, S, which):
    tab = model.casimir_table(synth.SPATIAL_ORBITAL, which)
    blocks, n, e, tasks = _setup(tab, LEFT_W, RIGHT_W, synth.SPATIAL_ORBITAL, N, S)
    psi = np.random.default_rng(1).standard_normal(n)
    F = heff.apply_heff(tab, e, tasks, blocks, n, psi)
    want = (S / 2) * (S / 2 + 1) if which == "S2" else N
    assert np.abs(F - want * psi).max() < 1e-13


def test_casimir_spin_chain():
    left = [(3, 1, 2), (3, 3, 1)]
    right = [(3, 1, 2), (3, 3, 1)]
    for S in (0, 2, 4):
        tab = model.casimir_table(synth.SPIN_HALF, "S2")
        blocks, n, e, tasks = _setup(tab, left, right, synth.SPIN_HALF, 8, S)
        psi = np.random.default_rng(2).standard_normal(n)
        F = heff.apply_heff(tab, e, tasks, blocks, n, psi)
        assert np.abs(F - (S / 2) * (S / 2 + 1) * psi).max() < 1e-13


@pytest.mark.parametrize("N,S", [(6, 0), (5, 1), (6, 2)])
def test_skeleton_against_mresolved_expansion(N, S):
    tab = model.qc_skeleton_table(2, 2)
    blocks, n, e, tasks = _setup(tab, LEFT, RIGHT, synth.SPATIAL_ORBITAL, N, S, seed=11)
    psi = np.random.default_rng(1).standard_normal(n)
    F = heff.apply_heff(tab, e, tasks, blocks, n, psi)
    G = expand.apply_heff_mresolved(tab, e, blocks, LEFT, RIGHT, S, psi)
    assert np.linalg.norm(F - G) <= 1e-12 * np.linalg.norm(F)


@pytest.mark.parametrize("N,S", [(6, 0), (5, 1)])
def test_skeleton_hermitian_and_diagonal(N, S):
    tab = model.qc_skeleton_table(2, 2)
    blocks, n, e, tasks = _setup(tab, LEFT_W, RIGHT_W, synth.SPATIAL_ORBITAL, N, S, seed=5)
    H = np.array([heff.apply_heff(tab, e, tasks, blocks, n, np.eye(n)[i]) for i in range(n)]).T
    assert np.abs(H - H.T).max() <= 1e-13 * np.abs(H).max()
    d = heff.diag_heff(tab, e, tasks, blocks, n)
    assert np.abs(d - np.diag(H)).max() <= 1e-14 * np.abs(H).max()


def test_planted_coupling_mistake_is_caught(monkeypatch):
    """Swapping the bra/ket roles in C~ (a plausible misreading of Eq. a)
    must break the agreement with the m-resolved expansion."""
    tab = model.qc_skeleton_table(2, 2)
    blocks, n, e, _ = _setup(tab, LEFT, RIGHT, synth.SPATIAL_ORBITAL, 5, 1, seed=11)
    psi = np.random.default_rng(1).standard_normal(n)
    G = expand.apply_heff_mresolved(tab, e, blocks, LEFT, RIGHT, 1, psi)
    good = su2.ctilde

    def swapped(j1, j2, j, k1, k2, k, j1p, j2p, jp):
        w = su2.ninej(j1, j2, j, k1, k2, k, j1p, j2p, jp)
        return math.sqrt((j1 + 1) * (j2 + 1) * (jp + 1) * (k + 1)) * w

    monkeypatch.setattr(heff, "ctilde", swapped)
    tasks = heff.build_tasks(tab, LEFT, RIGHT, blocks, 1)
    F = heff.apply_heff(tab, e, tasks, blocks, n, psi)
    assert np.linalg.norm(F - G) > 1e-3 * np.linalg.norm(G)
    monkeypatch.setattr(heff, "ctilde", good)


@pytest.mark.parametrize("L,D", [(6, 32), (8, 32), (8, 2), (10, 4)])
def test_heisenberg_against_full_projection(L, D):
    cfg = synth.Config("h", synth.SPIN_HALF, L, L, 0, D, 1001)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, synth.SPIN_HALF, L, 0)
    tab = model.heisenberg_table()
    e = env.build_env(tab, cfg, left, right)
    tasks = heff.build_tasks(tab, left, right, blocks, 0)
    psi = synth.gaussian_psi(n, 5)
    F = heff.apply_heff(tab, e, tasks, blocks, n, psi)
    G, P = expand.heisenberg_full_projection(cfg, blocks, left, right, psi)
    assert np.abs(P.T @ P - np.eye(n)).max() < 1e-13
    assert np.linalg.norm(F - G) <= 1e-13 * np.linalg.norm(F)


def test_heisenberg_l12_equals_exact_diagonalisation():
    cfg = synth.CONFIGS["heis12"]
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    # the full singlet sector of 12 spins has C(12,6)-C(12,5) = 132 states
    assert n == math.comb(12, 6) - math.comb(12, 5)
    tab = model.heisenberg_table()
    e = env.build_env(tab, cfg, left, right)
    tasks = heff.build_tasks(tab, left, right, blocks, cfg.twoS)
    d = heff.diag_heff(tab, e, tasks, blocks, n)
    th, x, res, it = davidson.davidson(lambda v: heff.apply_heff(tab, e, tasks, blocks, n, v), d,
                                       synth.gaussian_psi(n, synth.psi_seed(cfg)), tol=1e-10)
    E0 = ed.heisenberg_levels(12, 0)[0]
    assert res <= 1e-10
    assert abs(th - E0) < 1e-10


def test_ed_small_chains():
    # two sites: singlet -3/4; four sites: -(3/4 + sqrt(3)/2) ... closed form
    assert ed.heisenberg_levels(2, 0)[0] == pytest.approx(-0.75, abs=1e-14)
    assert ed.heisenberg_levels(4, 0)[0] == pytest.approx(-0.75 - math.sqrt(3) / 2, abs=1e-13)


def test_davidson_against_dense_eigensolver():
    tab = model.qc_skeleton_table(2, 2)
    blocks, n, e, tasks = _setup(tab, LEFT_W, RIGHT_W, synth.SPATIAL_ORBITAL, 6, 0, seed=9)
    H = np.array([heff.apply_heff(tab, e, tasks, blocks, n, np.eye(n)[i]) for i in range(n)]).T
    w = np.linalg.eigvalsh(0.5 * (H + H.T))
    d = heff.diag_heff(tab, e, tasks, blocks, n)
    th, x, res, it = davidson.davidson(lambda v: H @ v, d, synth.gaussian_psi(n, 3), tol=1e-10,
                                       max_sub=8)
    assert th == pytest.approx(w[0], abs=1e-10)


def test_weyl_paldus_matches_untruncated_chain():
    cfg = synth.Config("w", synth.SPATIAL_ORBITAL, 12, 12, 0, 10 ** 9, 1)
    chain = synth.bond_sector_chain(cfg, 6)
    for k, secs in enumerate(chain):
        for (n, s, d) in secs:
            assert d == synth.weyl_paldus(k, n, s)
        assert sum(d * (s + 1) for (_, s, d) in secs) == 4 ** k


def test_spin_chain_multiplets():
    cfg = synth.Config("w", synth.SPIN_HALF, 12, 12, 0, 10 ** 9, 1)
    chain = synth.bond_sector_chain(cfg, 8)
    for k, secs in enumerate(chain):
        for (n, s, d) in secs:
            assert d == synth.spin_chain_mult(k, s)
        assert sum(d * (s + 1) for (_, s, d) in secs) == 2 ** k
