"""The library's two-site sweep on the GPU (ab initio model and Heisenberg
chain, S = 0).

* Bonds that keep every multiplet: every window's energy is the full-CI
  ground-state energy (native FP64 and split paths).
* Truncated bonds: the energies of every window equal the oracle's sweep
  (its own SVD, truncation and renormalisation) on the same seeded MPS.
* Initial right blocks grown by the caller's MPS tensors.
* Wavefunction prediction: with bonds that keep every multiplet each
  predicted start vector is the eigenvector (one or two Davidson
  iterations); with truncated bonds the energies and the Rayleigh quotients
  of the predicted start vectors equal the oracle's predicted sweep.
* Checkpoint and resume: a sweep created from the right chain and MPS
  tensors checkpointed after one full sweep repeats the energies of the
  sweep that went on.
* The spin-1/2 Heisenberg chain (L = 12, D = 32, four sweeps): every window
  from the second half-sweep on equals exact diagonalisation; with D = 4
  the energies equal the oracle's sweep.
"""
import numpy as np
import pytest

import synth
from oracle import fci, sweep as osweep

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    torch.cuda.init()
    return P.Context(0, stream=torch.cuda.current_stream())


def lib_sweep(ctx, cfg, D, n_steps, prec):
    import paper_2309_16724_gb300 as P
    h, eri = synth.integrals(cfg.L, cfg.seed)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, h, eri, chain, cfg.N, D, prec=prec, tol=1e-10, seed=cfg.seed)
    e, w = sw.run(n_steps)
    sw.close()
    assert ctx.status() == 0
    return e, w


@pytest.mark.parametrize("prec", [0, 1])
def test_exact_sweep_equals_full_ci(ctx, prec):
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    e, w = lib_sweep(ctx, cfg, 400, 2 * (cfg.L - 1), prec)
    h, eri = synth.integrals(6, 1002)
    e0 = fci.spin_levels(h, eri, 6, 0)[0]
    assert np.abs(e - e0).max() < 1e-9
    assert np.all(np.abs(w) < 1e-20)


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_truncated_sweep_matches_oracle(ctx, prec, tol):
    cfg = synth.Config("sw7", synth.SPATIAL_ORBITAL, 7, 6, 0, 6, 1002)
    e, w = lib_sweep(ctx, cfg, 6, 2 * (cfg.L - 1), prec)
    eo, wo = osweep.sweep(cfg, 6, 2, tol=1e-10)
    assert len(e) == len(eo)
    assert np.abs(e - eo).max() < tol, (e, eo)
    wl = w[w > 0]
    assert np.allclose(np.sort(wl), np.sort(wo[wo > 0]), rtol=1e-6, atol=1e-12)


def test_sweep_from_caller_right_tensors(ctx):
    """The sweep's initial right blocks grown by the caller's tensors
    (random orthonormal, bonds that keep every multiplet): every window's
    energy is still full CI."""
    import paper_2309_16724_gb300 as P
    from test_lib_abinitio import random_tensors
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    h, eri = synth.integrals(6, 1002)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    _, flat = random_tensors(chain, np.random.default_rng(11))
    sw = P.Sweep(ctx, h, eri, chain, cfg.N, 400, prec=0, tol=1e-10, seed=cfg.seed, mps_right=flat)
    e, w = sw.run(2 * (cfg.L - 1))
    sw.close()
    assert ctx.status() == 0
    e0 = fci.spin_levels(h, eri, 6, 0)[0]
    assert np.abs(e - e0).max() < 1e-9


@pytest.mark.parametrize("prec", [0, 1])
def test_predicted_sweep_with_exact_bonds(ctx, prec):
    import paper_2309_16724_gb300 as P
    cfg = synth.Config("sw6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    h, eri = synth.integrals(6, 1002)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, h, eri, chain, cfg.N, 400, prec=prec, tol=1e-10, seed=cfg.seed, predict=True)
    e, w, it, e0 = sw.run(2 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    efci = fci.spin_levels(h, eri, 6, 0)[0]
    assert np.abs(e - efci).max() < 1e-9
    assert it[0] > 10 and it[1:].max() <= (2 if prec == 0 else 3), it
    assert np.abs(e0[1:] - efci).max() < 1e-9


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_predicted_sweep_matches_oracle(ctx, prec, tol):
    import paper_2309_16724_gb300 as P
    cfg = synth.Config("sw7", synth.SPATIAL_ORBITAL, 7, 6, 0, 6, 1002)
    h, eri = synth.integrals(cfg.L, cfg.seed)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, h, eri, chain, cfg.N, 6, prec=prec, tol=1e-10, seed=cfg.seed, predict=True)
    e, w, it, e0 = sw.run(2 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    so = []
    eo, wo = osweep.sweep(cfg, 6, 2, tol=1e-10, predict=True, stats=so)
    assert np.abs(e - eo).max() < tol, (e, eo)
    # the start vectors after the first window are the predicted ones on
    # both sides (the first is seeded differently)
    rq = np.array([x[1] for x in so])
    assert np.abs(e0[1:] - rq[1:]).max() < 1e-7, (e0, rq)
    assert it[cfg.L - 1] <= 2  # the turn starts from the previous eigenvector


@pytest.mark.parametrize("prec", [0, 1])
def test_heisenberg_sweep_c1_equals_exact_diagonalisation(ctx, prec):
    """The spin-1/2 Heisenberg chain, L = 12, D = 32, four sweeps from the
    seeded MPS with wavefunction prediction: from the second half-sweep on
    every window holds the exact ground state."""
    import paper_2309_16724_gb300 as P
    from oracle import ed
    cfg = synth.CONFIGS["heis12"]
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, None, None, chain, cfg.N, cfg.D, prec=prec, tol=1e-10, seed=cfg.seed, predict=True)
    e, w, it, e0 = sw.run(8 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    E0 = ed.heisenberg_levels(12, 0)[0]
    assert e.min() >= E0 - 1e-9
    assert np.abs(e[cfg.L - 1:] - E0).max() < 1e-9
    assert np.all(np.abs(w) < 1e-16)
    assert it[cfg.L - 1:].max() <= (2 if prec == 0 else 3), it


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_heisenberg_truncated_sweep_matches_oracle(ctx, prec, tol):
    import paper_2309_16724_gb300 as P
    cfg = synth.CONFIGS["heis12"]
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, None, None, chain, cfg.N, 4, prec=prec, tol=1e-10, seed=cfg.seed, predict=True)
    e, w, it, e0 = sw.run(4 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    so = []
    eo, wo = osweep.sweep(cfg, 4, 4, tol=1e-10, predict=True, stats=so)
    assert np.abs(e - eo).max() < tol, (e, eo)
    rq = np.array([x[1] for x in so])
    assert np.abs(e0[1:] - rq[1:]).max() < 1e-7, (e0, rq)
    wl = w[w > 0]
    assert np.allclose(np.sort(wl), np.sort(wo[wo > 0]), rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("model", ["abinitio", "heisenberg"])
def test_sweep_checkpoint_resumes(ctx, model):
    """A sweep resumed from the checkpoint taken after one full sweep (its
    right blocks' bond chain and MPS tensors) gives the same energies and
    discarded weights as the sweep that went on."""
    import paper_2309_16724_gb300 as P
    if model == "abinitio":
        cfg = synth.Config("sw7", synth.SPATIAL_ORBITAL, 7, 6, 0, 6, 1002)
        h, eri = synth.integrals(cfg.L, cfg.seed)
        D = 6
    else:
        cfg = synth.CONFIGS["heis12"]
        h = eri = None
        D = 6
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    a = P.Sweep(ctx, h, eri, chain, cfg.N, D, prec=0, tol=1e-10, seed=cfg.seed, predict=True)
    a.run(1)
    with pytest.raises(P.Su2Error):
        a.checkpoint()          # not at the start of a right-moving half-sweep
    a.run(2 * (cfg.L - 1) - 1)  # the rest of one full sweep: back at window 0
    rchain, mps = a.checkpoint()
    assert len(rchain) == cfg.L - 1 and mps.size > 0
    ea, wa = a.run(2 * (cfg.L - 1))
    a.close()
    b = P.Sweep(ctx, h, eri, rchain, cfg.N, D, prec=0, tol=1e-10, seed=cfg.seed, predict=True, mps_right=mps)
    eb, wb = b.run(2 * (cfg.L - 1))
    b.close()
    assert ctx.status() == 0
    assert np.abs(ea - eb).max() < 1e-8, (ea, eb)
    assert np.allclose(wa, wb, rtol=1e-5, atol=1e-12)


@pytest.mark.parametrize("N,twoS", [(5, 1), (6, 2)])
def test_spin_target_sweep_equals_full_ci(ctx, N, twoS):
    """Targets with S > 0 (bond matrices over every j_2R, prediction
    recoupled by a 6j), bonds that keep every multiplet: every window equals
    the lowest spin-S level of full CI, after the first window in one or
    two iterations."""
    import paper_2309_16724_gb300 as P
    cfg = synth.Config("sws", synth.SPATIAL_ORBITAL, 6, N, twoS, 400, 1002)
    h, eri = synth.integrals(6, 1002)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, h, eri, chain, N, 400, prec=0, tol=1e-10, seed=cfg.seed, predict=True, twoS=twoS)
    e, w, it, e0 = sw.run(2 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    assert np.abs(e - fci.spin_levels(h, eri, N, twoS)[0]).max() < 1e-9
    assert it[1:].max() <= 2, it


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-8)])
def test_spin_target_truncated_sweep_matches_oracle(ctx, prec, tol):
    import paper_2309_16724_gb300 as P
    cfg = synth.Config("sw7s1", synth.SPATIAL_ORBITAL, 7, 6, 2, 6, 1002)
    h, eri = synth.integrals(cfg.L, cfg.seed)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, h, eri, chain, cfg.N, 6, prec=prec, tol=1e-10, seed=cfg.seed, predict=True, twoS=2)
    e, w, it, e0 = sw.run(2 * (cfg.L - 1), stats=True)
    sw.close()
    assert ctx.status() == 0
    so = []
    eo, wo = osweep.sweep(cfg, 6, 2, tol=1e-10, predict=True, stats=so)
    assert np.abs(e - eo).max() < tol, (e, eo)
    rq = np.array([x[1] for x in so])
    assert np.abs(e0[1:] - rq[1:]).max() < 1e-7, (e0, rq)


def test_heisenberg_triplet_sweep_equals_exact_diagonalisation(ctx):
    import paper_2309_16724_gb300 as P
    from oracle import ed
    cfg = synth.Config("h10s1", synth.SPIN_HALF, 10, 10, 2, 32, 1001)
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    sw = P.Sweep(ctx, None, None, chain, cfg.N, 32, prec=1, tol=1e-10, seed=cfg.seed, predict=True, twoS=2)
    e, w = sw.run(4 * (cfg.L - 1))
    sw.close()
    assert ctx.status() == 0
    E0 = ed.heisenberg_levels(10, 2)[0]
    assert e.min() >= E0 - 1e-9
    assert np.abs(e[cfg.L - 1:] - E0).max() < 1e-9
