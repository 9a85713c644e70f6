"""Pins of the oracle's two-site sweep (Sec. II) on the ab initio Hamiltonian.

* With bonds that keep every multiplet, every step's Davidson energy is the
  full-CI ground-state energy (the two-site space is then the whole
  N-electron spin-0 space).
* With truncated bonds the energies are variational (never below full CI)
  and the discarded weights are non-negative.
* The SVD isometries: kept columns are orthonormal, the kept sectors hold at
  most D multiplets, and with D large enough nothing is discarded and the
  bond matrices are reproduced.
* Wavefunction prediction: the predicted start vector of the next window is
  the truncated state written in that window's basis (its norm and its
  Rayleigh quotient are those of the truncated state, for any vector and
  any truncation); with exact bonds it is the converged eigenvector; a
  right block expanded with a wrong tensor breaks the identity.
* The spin-1/2 Heisenberg chain (L = 12, D = 32, four sweeps): every window
  from the second half-sweep on equals exact diagonalisation; with D = 4 the
  energies are variational.
* Targets with S > 0 (S = 1/2, 1): exact sweeps equal full CI and exact
  diagonalisation, the prediction (which recouples by a 6j) keeps the
  truncated-state identities, and the S = 0 factor planted in its place
  breaks them.
"""
import numpy as np
import pytest

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


_SW7 = synth.Config("sw7", synth.SPATIAL_ORBITAL, 7, 6, 0, 6, 1002)
_SW7_RUNS = {}


def _sw7(predict):
    """Two half-sweeps of the seven-orbital chain at D = 6 (run once per
    flag and shared by the tests): (energies, discarded weights, stats)."""
    if predict not in _SW7_RUNS:
        st = []
        E, w = sweep.sweep(_SW7, 6, 2, predict=predict, stats=st)
        _SW7_RUNS[predict] = (E, w, st)
    return _SW7_RUNS[predict]


def test_truncated_sweep_is_variational():
    cfg = _SW7
    E, w, _ = _sw7(False)
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


# ---------------------------------------------------------------- wavefunction prediction
# The predicted start vector of the next window is the truncated state of
# the previous one written in the next window's basis, so (for any vector,
# converged or not) its squared norm is 1 - discarded weight and its
# Rayleigh quotient in the next window equals that of the truncated state in
# the window it came from.  Both windows' H_eff are projections P^T H P of
# the same Hamiltonian onto spaces that contain that state.

def _from_bond_matrices(mats, blocks, n, side):
    """Inverse of the bond-matrix view (``sweep._bond_matrices``'s layout)
    back into the flat two-site vector."""
    out = np.zeros(n)
    bidx = sectors.block_index(blocks)
    for (Nk, j), (rows, cols, M) in mats.items():
        if side == "L":
            for (a, s1, r0, da) in rows:
                for (jo, b, s2, c0, db) in cols:
                    sectors.block_view(out, blocks[bidx[(a, s1, s2, b, j, jo)]])[:] = M[r0:r0 + da, c0:c0 + db]
        else:
            for (jo, a, s1, r0, da) in rows:
                for (b, s2, c0, db) in cols:
                    sectors.block_view(out, blocks[bidx[(a, s1, s2, b, jo, j)]])[:] = M[r0:r0 + da, c0:c0 + db]
    return out


def _truncated(psi, blocks, n, ls, rs, N, sec, A, rest, side, kind=synth.SPATIAL_ORBITAL, twoS=0):
    mats = sweep._bond_matrices(psi, blocks, ls, rs, kind, N, twoS, side)
    kept = {}
    for qo, (Nb, j, d) in enumerate(sec):
        rows, cols, M = mats[(Nb, j)]
        Q, C = A[qo][1], rest[qo][1]
        kept[(Nb, j)] = (rows, cols, Q @ C if side == "L" else C @ Q.T)
    for key, (rows, cols, M) in mats.items():
        if key not in kept:
            kept[key] = (rows, cols, np.zeros_like(M))
    return _from_bond_matrices(kept, blocks, n, side)


def _rq(apply, v):
    return float(v @ apply(v) / (v @ v))


def _prediction_chain(L, N, D, seed, plant=None, twoS=0):
    """Walks windows 0 .. L-2 moving right and back moving left with seeded
    (unconverged) vectors, growing blocks with the truncated isometries;
    returns per transition (|guess|^2, 1 - w, RQ of the guess in the next
    window, RQ of the truncated state in its own window)."""
    from oracle import abinitio
    from oracle import env as envmod
    kind = synth.SPATIAL_ORBITAL
    cfg = synth.Config("pred", kind, L, N, twoS, D, seed)
    h, eri = synth.integrals(L, seed)
    strings = abinitio.hamiltonian_strings(h, eri)
    chain = synth.bond_sector_chain(cfg, L - 2)
    R, RA = [abinitio.RightBlock(strings, L)], [None] * (L - 1)
    for k in range(1, L - 1):
        RA[k] = envmod.mps_tensor(seed, envmod.SIDE_MPS_R, k, chain[k - 1], chain[k], kind)
        R.append(R[-1].grown(chain[k], RA[k]))
    Lbs, LA = [abinitio.LeftBlock(strings, L)] + [None] * (L - 2), [None] * (L - 1)
    out = []
    for i in range(0, L - 2):
        apply, _, blocks, n, ls, rs = sweep.window(strings, Lbs[i], R[L - 2 - i], N, twoS)
        psi = synth.gaussian_psi(n, 50 + i)
        sec, A, w, rest = sweep.isometry(psi, blocks, ls, rs, kind, N, D, "L", with_rest=True, twoS=twoS)
        Lbs[i + 1] = Lbs[i].grown(sec, A)
        LA[i + 1] = A
        apply2, _, nb, nn, _, _ = sweep.window(strings, Lbs[i + 1], R[L - 3 - i], N, twoS)
        RAi = RA[L - 2 - i] if plant is None else plant(RA[L - 2 - i])
        g = sweep.predict_moving_right(rest, rs, RAi, nb, nn, sec, twoS, kind)
        t = _truncated(psi, blocks, n, ls, rs, N, sec, A, rest, "L", kind, twoS)
        out.append((g @ g, 1.0 - w, _rq(apply2, g), _rq(apply, t)))
    for i in range(L - 2, 0, -1):
        apply, _, blocks, n, ls, rs = sweep.window(strings, Lbs[i], R[L - 2 - i], N, twoS)
        psi = synth.gaussian_psi(n, 80 + i)
        sec, A, w, rest = sweep.isometry(psi, blocks, ls, rs, kind, N, D, "R", with_rest=True, twoS=twoS)
        R[L - 1 - i] = R[L - 2 - i].grown(sec, A)
        RA[L - 1 - i] = A
        apply2, _, nb, nn, _, _ = sweep.window(strings, Lbs[i - 1], R[L - 1 - i], N, twoS)
        g = sweep.predict_moving_left(rest, ls, LA[i], nb, nn, sec, twoS, kind)
        t = _truncated(psi, blocks, n, ls, rs, N, sec, A, rest, "R", kind, twoS)
        out.append((g @ g, 1.0 - w, _rq(apply2, g), _rq(apply, t)))
    return out


def test_prediction_is_the_truncated_state_in_the_next_window():
    # D = 5 truncates every inner bond of the seven-orbital chain
    res = _prediction_chain(7, 6, 5, 1003)
    assert len(res) == 2 * 5
    assert max(1.0 - w for (_, w, _, _) in res) > 1e-3     # weight was discarded
    for (g2, w, e_next, e_trunc) in res:
        assert abs(g2 - w) <= 1e-12
        assert abs(e_next - e_trunc) <= 1e-11 * abs(e_trunc)


def test_prediction_with_a_wrong_right_tensor_fails():
    # a planted mistake: the right block expanded with its tensor's columns
    # in the wrong order (still an isometry, a different state)
    def swap(RA):
        out = {}
        for b, (rows, G) in RA.items():
            out[b] = (rows, G[:, ::-1].copy())
        return out
    res = _prediction_chain(6, 6, 5, 1003, plant=swap)
    assert max(abs(e - t) for (_, _, e, t) in res[:4]) > 1e-4


def test_prediction_with_exact_bonds_is_an_eigenvector():
    # bonds keep every multiplet: the converged vector of window 1, predicted
    # into window 2, is the same eigenstate
    from oracle import abinitio, davidson
    from oracle import env as envmod
    L, N, seed = 6, 6, 1002
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, L, N, 0, 400, seed)
    h, eri = synth.integrals(L, seed)
    strings = abinitio.hamiltonian_strings(h, eri)
    chain = synth.bond_sector_chain(cfg, L - 2)
    R, RA = [abinitio.RightBlock(strings, L)], [None] * (L - 1)
    for k in range(1, L - 1):
        RA[k] = envmod.mps_tensor(seed, envmod.SIDE_MPS_R, k, chain[k - 1], chain[k], synth.SPATIAL_ORBITAL)
        R.append(R[-1].grown(chain[k], RA[k]))
    Lb = abinitio.LeftBlock(strings, L)
    apply, diag, blocks, n, ls, rs = sweep.window(strings, Lb, R[L - 2], N)
    theta, x, res, _ = davidson.davidson(apply, diag, synth.gaussian_psi(n, 3), tol=1e-11)
    sec, A, w, rest = sweep.isometry(x, blocks, ls, rs, synth.SPATIAL_ORBITAL, N, 400, "L", with_rest=True)
    assert abs(w) < 1e-20
    Lb1 = Lb.grown(sec, A)
    apply2, _, nb, nn, _, _ = sweep.window(strings, Lb1, R[L - 3], N)
    g = sweep.predict_moving_right(rest, rs, RA[L - 2], nb, nn)
    assert abs(np.linalg.norm(g) - 1.0) < 1e-12
    assert np.linalg.norm(apply2(g) - theta * g) < 1e-9
    assert abs(theta - fci.spin_levels(h, eri, N, 0)[0]) < 1e-9


def test_predicted_sweep_same_energies_fewer_iterations():
    # exact bonds: after the first window every predicted start vector is the
    # converged eigenvector, so Davidson stops after its first iteration
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    st = []
    E, w = sweep.sweep(cfg, 400, 2, predict=True, stats=st)
    h, eri = synth.integrals(6, 1002)
    assert np.abs(E - fci.spin_levels(h, eri, 6, 0)[0]).max() < 1e-9
    assert st[0][0] > 10 and all(it == 1 for (it, _) in st[1:])
    # truncated bonds: the same energies and discarded weights as the sweep
    # from seeded start vectors, in fewer iterations
    cfg = _SW7
    E0, w0, s0 = _sw7(False)
    E1, w1, s1 = _sw7(True)
    assert np.abs(E1 - E0).max() < 1e-8
    assert np.abs(w1 - w0).max() < 1e-8
    assert sum(s[0] for s in s1) < sum(s[0] for s in s0)
    # the turn's start vector is the previous window's eigenvector
    assert s1[cfg.L - 1][0] == 1


# ---------------------------------------------------------------- Heisenberg chain
def test_heisenberg_sweep_c1_equals_exact_diagonalisation():
    # L = 12, D = 32, four sweeps from the seeded MPS: the initial right
    # blocks are truncated (up to 252 multiplets per bond), but the ground
    # state's bonds hold at most 20 multiplets, so from the second half-sweep
    # on every window holds the exact ground state
    from oracle import ed
    cfg = synth.CONFIGS["heis12"]
    E0 = ed.heisenberg_levels(12, 0)[0]
    for predict in (False, True):
        st = []
        E, w = sweep.sweep(cfg, 32, 8, tol=1e-10, predict=predict, stats=st)
        assert len(E) == 8 * (cfg.L - 1)
        assert E.min() >= E0 - 1e-10
        assert np.abs(E[cfg.L - 1:] - E0).max() < 1e-9
        assert np.all(np.abs(w) < 1e-20)
        if predict:
            assert all(it == 1 for (it, _) in st[cfg.L - 1:])


def test_heisenberg_truncated_sweep_is_variational():
    from oracle import ed
    cfg = synth.CONFIGS["heis12"]
    E0 = ed.heisenberg_levels(12, 0)[0]
    E, w = sweep.sweep(cfg, 4, 8, tol=1e-10)
    assert E.min() >= E0 - 1e-12 and w.max() > 0
    # the last sweep is within its truncation error of the ground state
    assert np.all(E[-(cfg.L - 1):] - E0 < 1e-4)
    assert abs(E[cfg.L - 2] - E[cfg.L - 1]) < 1e-9


# ---------------------------------------------------------------- targets with S > 0
@pytest.mark.parametrize("N,twoS", [(5, 1), (6, 2)])
def test_prediction_for_spin_targets_is_the_truncated_state(N, twoS):
    # at S > 0 the guess recouples [k x (s2 x b)_j2R]^S by a 6j; the
    # identities of the truncated state still hold to rounding
    res = _prediction_chain(6, N, 5, 1003, twoS=twoS)
    assert max(1.0 - w for (_, w, _, _) in res) > 1e-3
    for (g2, w, e_next, e_trunc) in res:
        assert abs(g2 - w) <= 1e-12
        assert abs(e_next - e_trunc) <= 1e-11 * abs(e_trunc)


def test_prediction_without_the_recoupling_fails(monkeypatch):
    # a planted mistake: the S = 0 factor (1) used for an S = 1 target
    monkeypatch.setattr(sweep, "_recouple", lambda *a: 1.0)
    res = _prediction_chain(6, 6, 5, 1003, twoS=2)
    assert max(abs(e - t) / abs(t) for (_, _, e, t) in res) > 1e-3


@pytest.mark.parametrize("N,twoS", [(5, 1), (6, 2)])
def test_exact_sweep_for_spin_targets_equals_full_ci(N, twoS):
    cfg = synth.Config("sws", synth.SPATIAL_ORBITAL, 6, N, twoS, 400, 1002)
    st = []
    E, w = sweep.sweep(cfg, 400, 2, predict=True, stats=st)
    h, eri = synth.integrals(6, 1002)
    assert np.abs(E - fci.spin_levels(h, eri, N, twoS)[0]).max() < 1e-9
    assert np.all(np.abs(w) < 1e-20)
    assert all(it == 1 for (it, _) in st[1:])


def test_heisenberg_triplet_sweep_equals_exact_diagonalisation():
    from oracle import ed
    cfg = synth.Config("h10s1", synth.SPIN_HALF, 10, 10, 2, 32, 1001)
    E, w = sweep.sweep(cfg, 32, 4, tol=1e-10, predict=True)
    E0 = ed.heisenberg_levels(10, 2)[0]
    assert E.min() >= E0 - 1e-10
    assert np.abs(E[cfg.L - 1:] - E0).max() < 1e-9
