"""Pins of the ab initio oracle (Eq. 1 in the normal/complementary partition).

* full CI against closed forms (one orbital; no two-body part);
* the seeded integrals have the stated symmetries and positivity;
* the generic site-operator reduction reproduces the reduced site operators
  of Sec. II.B;
* with bond dimensions that keep every multiplet, H_eff's spectrum equals
  the spin-S levels of the N-electron full CI (S = 0, 1/2, 1; even and odd N)
  and its dimension the Weyl-Paldus count;
* the two-site block enumeration agrees with an independent multiplicity
  count by characters on truncated bonds;
* H_eff is symmetric with truncated bonds, and equals P^T H P elementwise,
  P the two-site basis built as explicit vectors of the determinant space
  from the same seeded MPS and H the full-CI matrix (full and truncated
  bonds, S = 0, 1/2, 1);
* a planted sign error in the oracle's annihilator convention breaks the
  full-CI agreement (the pin has teeth).
"""
import numpy as np
import pytest

import synth
from oracle import abinitio, fci, heff, sectors
from oracle import model as omodel


def dense_heff(cfg, h=None, eri=None):
    table, env, lsec, rsec = abinitio.build_problem(cfg, h, eri)
    left, right = synth.middle_bond_sectors(cfg)
    assert (left, right) == (lsec, rsec)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    tasks = heff.build_tasks(table, left, right, blocks, cfg.twoS)
    return np.array([heff.apply_heff(table, env, tasks, blocks, n, np.eye(n)[i]) for i in range(n)]).T


def test_fci_one_orbital_closed_form():
    h = np.array([[-1.3]])
    eri = np.array([[[[0.7]]]])
    H, _ = fci.hamiltonian_sector(h, eri, 2, 0)
    assert H.shape == (1, 1)
    assert abs(H[0, 0] - (2 * -1.3 + 0.7)) < 1e-14
    H1, _ = fci.hamiltonian_sector(h, eri, 1, 1)
    assert abs(H1[0, 0] + 1.3) < 1e-14


def test_fci_one_body_closed_form():
    L = 5
    h, _ = synth.integrals(L, 7)
    eri = np.zeros((L, L, L, L))
    eps = np.linalg.eigvalsh(h)
    for N in (2, 4, 6):
        e0 = np.linalg.eigvalsh(fci.hamiltonian_sector(h, eri, N, 0)[0])[0]
        assert abs(e0 - 2 * eps[: N // 2].sum()) < 1e-12
    # odd N, S_z = 1/2: the extra electron in the next orbital
    e0 = np.linalg.eigvalsh(fci.hamiltonian_sector(h, eri, 3, 1)[0])[0]
    assert abs(e0 - (2 * eps[0] + eps[1])) < 1e-12


def test_fci_hermitian_and_spin_levels_count():
    h, eri = synth.integrals(5, 11)
    H, st = fci.hamiltonian_sector(h, eri, 5, 1)
    assert np.abs(H - H.T).max() < 1e-13
    lev = fci.spin_levels(h, eri, 5, 1)
    assert len(lev) == synth.weyl_paldus(5, 5, 1)


def test_integrals_symmetry_and_positivity():
    L = 9
    h, eri = synth.integrals(L, 1002)
    assert np.allclose(h, h.T)
    assert (np.diag(h) >= -2).all() and (np.diag(h) <= 0).all()
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.allclose(eri, eri.transpose(perm))
    assert np.linalg.eigvalsh(eri.reshape(L * L, L * L)).min() > -1e-12
    # the off-diagonal decay exp(-|i-j|/4) of the recipe: the far corner is
    # e^{-2} times a standard-normal-sized number
    assert abs(h[0, L - 1]) < 5 * np.exp(-(L - 1) / 4)
    # reproducible
    h2, eri2 = synth.integrals(L, 1002)
    assert np.array_equal(h, h2) and np.array_equal(eri, eri2)


def test_generic_site_operators_match_sec2b():
    ref = omodel.site_ops(synth.SPATIAL_ORBITAL)
    C, A = abinitio.CREATE, abinitio.ANNIHILATE
    assert np.allclose(abinitio.site_op((C,), ()).mat(), ref["cdag"].mat())
    assert np.allclose(abinitio.site_op((A,), ()).mat(), ref["c"].mat())
    # n = sum_s c+_s c_s = -sqrt(2) [a+ x a~]^0
    assert np.allclose(-np.sqrt(2) * abinitio.site_op((C, A), (0,)).mat(), ref["n"].mat())
    # pair = [a+ x a+]^0 = sqrt(2) c+_up c+_dn
    assert np.allclose(abinitio.site_op((C, C), (0,)).mat(), ref["pair"].mat())
    assert abinitio.site_op((C, C), (2,)) is None        # [a+ x a+]^1 = 0 on one orbital


@pytest.mark.parametrize("L,N,twoS", [(4, 4, 0), (6, 6, 0), (6, 5, 1), (6, 4, 2), (6, 7, 1)])
def test_heff_spectrum_equals_full_ci(L, N, twoS):
    cfg = synth.Config("fci", synth.SPATIAL_ORBITAL, L, N, twoS, 400, 1002)
    Hm = dense_heff(cfg)
    assert np.abs(Hm - Hm.T).max() < 1e-12
    ev = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))
    h, eri = synth.integrals(L, 1002)
    ref = fci.spin_levels(h, eri, N, twoS)
    assert len(ev) == len(ref) == synth.weyl_paldus(L, N, twoS)
    assert np.abs(ev - ref).max() < 1e-11


def _mult_by_characters(spins, S):
    """Multiplicity of spin S in the product of spins (twos), by counting
    states with M = S and M = S + 1."""
    counts = {0: 1}
    for j in spins:
        new = {}
        for M, c in counts.items():
            for m in range(-j, j + 1, 2):
                new[M + m] = new.get(M + m, 0) + c
        counts = new
    return counts.get(S, 0) - counts.get(S + 2, 0)


@pytest.mark.parametrize("L,N,twoS,D", [(10, 10, 0, 40), (12, 11, 1, 60), (16, 16, 0, 512)])
def test_block_enumeration_by_characters(L, N, twoS, D):
    cfg = synth.Config("enum", synth.SPATIAL_ORBITAL, L, N, twoS, D, 3)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, N, twoS)
    site = synth.site_states(cfg.site_kind)
    want = 0
    for (Na, Sa, da) in left:
        for (n1, t1) in site:
            for (n2, t2) in site:
                for (Nb, Sb, db) in right:
                    if Na + n1 + n2 + Nb == N:
                        want += da * db * _mult_by_characters([Sa, t1, t2, Sb], twoS)
    assert n == want == sum(B.rows * B.cols for B in blocks)


def test_full_bonds_enumerate_all_multiplets():
    for (L, N, twoS) in [(6, 6, 0), (8, 7, 1), (8, 8, 2)]:
        cfg = synth.Config("full", synth.SPATIAL_ORBITAL, L, N, twoS, 10 ** 6, 3)
        left, right = synth.middle_bond_sectors(cfg)
        _, n = sectors.build_blocks(left, right, cfg.site_kind, N, twoS)
        assert n == synth.weyl_paldus(L, N, twoS)


def test_heff_symmetric_with_truncated_bonds():
    cfg = synth.Config("trunc", synth.SPATIAL_ORBITAL, 10, 9, 1, 30, 1002)
    table, env, _, _ = abinitio.build_problem(cfg)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    tasks = heff.build_tasks(table, left, right, blocks, cfg.twoS)
    psi, phi = synth.gaussian_psi(n, 1), synth.gaussian_psi(n, 2)
    Hp = heff.apply_heff(table, env, tasks, blocks, n, psi)
    Hf = heff.apply_heff(table, env, tasks, blocks, n, phi)
    assert abs(phi @ Hp - psi @ Hf) <= 1e-13 * np.linalg.norm(Hp)


def test_planted_annihilator_sign_error_is_caught(monkeypatch):
    """Flip the sign of the spin-down annihilator component in the oracle's
    Hamiltonian tensors: the spectrum must no longer match full CI."""
    def bad_one_body():
        F = np.zeros((2, 2))
        for s in (0, 1):
            F[s, 1 - s] = -1.0
        return F
    abinitio.site_op.cache_clear()
    monkeypatch.setattr(abinitio, "_one_body_tensor", bad_one_body)
    cfg = synth.Config("fci", synth.SPATIAL_ORBITAL, 4, 4, 0, 400, 1002)
    Hm = dense_heff(cfg)
    ev = np.linalg.eigvalsh(0.5 * (Hm + Hm.T))
    h, eri = synth.integrals(4, 1002)
    ref = fci.spin_levels(h, eri, 4, 0)
    assert np.abs(ev - ref).max() > 1e-3


@pytest.mark.parametrize("L,N,twoS,D", [(6, 6, 0, 6), (6, 5, 1, 5), (6, 6, 2, 4), (7, 6, 0, 8)])
def test_heff_equals_explicit_projection(L, N, twoS, D):
    """H_eff of the normal/complementary construction equals P^T H P with
    the block bases written out as determinant-space vectors (Clebsch-Gordan
    couplings of the seeded MPS, no 6j or 9j, no renormalised operators),
    on truncated bonds too, where full CI alone would not pin it."""
    from oracle import expand
    cfg = synth.Config("proj", synth.SPATIAL_ORBITAL, L, N, twoS, D, 1002)
    He = dense_heff(cfg)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, N, twoS)
    h, eri = synth.integrals(L, cfg.seed)
    Hp, P = expand.abinitio_full_projection(cfg, blocks, n, h, eri)
    assert np.abs(P.T @ P - np.eye(n)).max() < 1e-13
    assert np.abs(He - Hp).max() <= 1e-12 * np.abs(He).max()
