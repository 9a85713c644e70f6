"""The ab initio Hamiltonian (Eq. 1 from the seeded integrals) on the GPU.

The environment is built on the device: the block operators are
renormalised orbital by orbital through the grouped FP64 kernels.  Checked
against the oracle (its own normal/complementary construction, pinned by
full CI):

* the renormalised block Hamiltonians H_L, H_R block by block (<= 1e-12);
* H.psi at L = N = 16, D = 512: native FP64 (<= 1e-12) and split BF16
  (<= 1e-10) against the oracle, elementwise as well;
* Davidson on a chain whose bonds keep every multiplet: the ground-state
  energy equals full CI (FP64 and split paths);
* Davidson at L = N = 16, D = 512: split and FP64 energies within 1e-9;
* the device-built and host-built operators agree.
"""
import numpy as np
import pytest

import synth
from oracle import abinitio, fci, heff, sectors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    torch.cuda.init()
    return P.Context(0, stream=torch.cuda.current_stream())


@pytest.fixture(scope="module")
def qc16(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc16"]
    sec, env = workload.build(ctx, cfg, model=P.SU2_MODEL_AB_INITIO, prepare_split=True, n_slices=5)
    table, oenv, lsec, rsec = abinitio.build_problem(cfg)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = sectors.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    tasks = heff.build_tasks(table, left, right, blocks, cfg.twoS)
    return dict(cfg=cfg, sec=sec, env=env, oenv=oenv, lsec=lsec, rsec=rsec,
                oapply=lambda psi: heff.apply_heff(table, oenv, tasks, blocks, n, psi))


def gpu_apply(ctx, env, psi, prec):
    import paper_2309_16724_gb300 as P
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    P.apply_heff(ctx, env, x, y, prec)
    torch.cuda.synchronize()
    assert ctx.status() == 0
    return y.cpu().numpy()


def test_gpu_renormalised_block_hamiltonians(qc16):
    env, oenv = qc16["env"], qc16["oenv"]
    assert env.info["renorm_flops"] > 1e10
    for side, name, S in ((0, "L", qc16["lsec"]), (1, "R", qc16["rsec"])):
        nb = 0
        for (qo, qi), M in oenv[(name, 1)].items():
            Mb = env.operator_block(side, 1, qo, qi, S[qo][2], S[qi][2])
            assert np.abs(Mb - M).max() <= 1e-12 * max(1.0, np.abs(M).max())
            nb += 1
        assert nb >= 10


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-10)])
def test_qc16_from_integrals_matches_oracle(ctx, qc16, prec, tol):
    psi = synth.gaussian_psi(qc16["sec"].psi_len, synth.psi_seed(qc16["cfg"]))
    F = qc16["oapply"](psi)
    G = gpu_apply(ctx, qc16["env"], psi, prec)
    assert np.linalg.norm(G - F) <= tol * np.linalg.norm(F)
    assert np.abs(G - F).max() <= tol * np.abs(F).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_davidson_equals_full_ci(ctx, prec):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("fci6", synth.SPATIAL_ORBITAL, 6, 6, 0, 400, 1002)
    sec, env = workload.build(ctx, cfg, model=P.SU2_MODEL_AB_INITIO, prepare_split=prec == 1, n_slices=5)
    psi0 = torch.from_numpy(synth.gaussian_psi(sec.psi_len, 7)).cuda()
    dav = P.Davidson(ctx, env, psi0, tol=1e-9, prec=prec)
    th, res, it, ok = dav.solve()
    assert ok
    h, eri = synth.integrals(6, 1002)
    e0 = fci.spin_levels(h, eri, 6, 0)[0]
    assert abs(th - e0) <= 1e-9


def test_davidson_split_energy_matches_fp64_qc16(ctx, qc16):
    import paper_2309_16724_gb300 as P
    env = qc16["env"]
    psi0 = torch.from_numpy(synth.gaussian_psi(qc16["sec"].psi_len, 17)).cuda()
    th = {}
    for prec in (0, 1):
        dav = P.Davidson(ctx, env, psi0, tol=1e-8, prec=prec, max_iter=400)
        t, res, it, ok = dav.solve()
        assert ok, (prec, res, it)
        th[prec] = t
        dav.close()
    assert abs(th[1] - th[0]) <= 1e-9


def test_device_and_host_built_operators_agree(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("ab10", synth.SPATIAL_ORBITAL, 10, 10, 0, 60, 1002)
    hctx = P.Context(-1)
    sec_d, env_d = workload.build(ctx, cfg, model=P.SU2_MODEL_AB_INITIO)
    sec_h, env_h = workload.build(hctx, cfg, model=P.SU2_MODEL_AB_INITIO)
    assert env_d.info["n_terms"] == env_h.info["n_terms"] and env_d.info["n_tasks"] == env_h.info["n_tasks"]
    ad, dd, _, _ = env_d.terms()
    for side, S in ((0, sec_d.left), (1, sec_d.right)):
        ops = set((ad if side == 0 else dd).tolist()) - {0}
        for op in sorted(ops)[:40]:
            for qo in range(len(S)):
                for qi in range(len(S)):
                    try:
                        a = env_d.operator_block(side, op, qo, qi, S[qo][2], S[qi][2])
                    except P.Su2Error:
                        continue
                    b = env_h.operator_block(side, op, qo, qi, S[qo][2], S[qi][2])
                    assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(b).max())
    env_h.close()
    hctx.close()
