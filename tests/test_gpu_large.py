"""Full-size checks at the benchmark configuration (qc32: L=N=32, S=0,
D=2048, the launch configuration bench.py times), on sampled output blocks
that the oracle computes one by one, plus properties that hold at any size;
and Davidson energies of the split path against the FP64 path.
"""
import numpy as np
import pytest

import synth
from oracle import env as oenv
from oracle import heff as oheff
from oracle import model as omodel
from oracle import sectors as osec

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    return P.Context(0, stream=torch.cuda.current_stream())


@pytest.fixture(scope="module")
def qc32(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc32"]
    sec, env = workload.build(ctx, cfg, prepare_split=True)
    psi = synth.gaussian_psi(sec.psi_len, synth.psi_seed(cfg))
    x = torch.from_numpy(psi).cuda()
    y64 = torch.empty_like(x)
    ysp = torch.empty_like(x)
    P.apply_heff(ctx, env, x, y64, P.SU2_FP64)
    P.apply_heff(ctx, env, x, ysp, P.SU2_SPLIT_BF16)
    assert ctx.status() == 0
    return dict(cfg=cfg, sec=sec, env=env, psi=psi, f64=y64.cpu().numpy(), split=ysp.cpu().numpy())


def test_split_vs_fp64_full_vector(qc32):
    a, b = qc32["split"], qc32["f64"]
    assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def test_sampled_blocks_against_oracle(qc32):
    cfg = qc32["cfg"]
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    assert n == qc32["sec"].psi_len
    order = sorted(range(len(blocks)), key=lambda f: -blocks[f].rows * blocks[f].cols)
    rng = np.random.default_rng(7)
    # the largest block, a median one, the smallest (ragged) one and a random one
    sel = {order[0], order[len(order) // 2], order[-1], int(rng.integers(len(blocks)))}
    tab = omodel.qc_skeleton_table(cfg.n_left, cfg.n_right)
    e = oenv.LazySyntheticEnv(tab, cfg, left, right)
    tasks = oheff.build_tasks(tab, left, right, blocks, cfg.twoS, only_f=sel)
    F = oheff.apply_heff(tab, e, tasks, blocks, n, qc32["psi"])
    idx = np.concatenate([np.arange(blocks[f].offset, blocks[f].offset + blocks[f].rows * blocks[f].cols)
                          for f in sorted(sel)])
    ref = F[idx]
    assert np.linalg.norm(qc32["f64"][idx] - ref) <= 1e-12 * np.linalg.norm(ref)
    assert np.linalg.norm(qc32["split"][idx] - ref) <= 1e-10 * np.linalg.norm(ref)


def test_hermiticity_full_size(ctx, qc32):
    import paper_2309_16724_gb300 as P
    phi = synth.gaussian_psi(qc32["sec"].psi_len, 99)
    x = torch.from_numpy(phi).cuda()
    y = torch.empty_like(x)
    P.apply_heff(ctx, qc32["env"], x, y, P.SU2_SPLIT_BF16)
    torch.cuda.synchronize()
    Hphi = y.cpu().numpy()
    lhs = phi @ qc32["split"]
    rhs = Hphi @ qc32["psi"]
    assert abs(lhs - rhs) <= 1e-10 * np.linalg.norm(qc32["split"]) * np.linalg.norm(phi)


def test_davidson_split_energy_matches_fp64(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("qc12D100", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 9)
    sec, env = workload.build(ctx, cfg, prepare_split=True)
    psi0 = torch.from_numpy(synth.gaussian_psi(sec.psi_len, synth.psi_seed(cfg))).cuda()
    res = {}
    for prec in (P.SU2_FP64, P.SU2_SPLIT_BF16):
        dav = P.Davidson(ctx, env, psi0, tol=1e-7, prec=prec, max_iter=300)
        th, r, it, ok = dav.solve()
        assert ok, (prec, th, r, it)
        res[prec] = th
    assert abs(res[P.SU2_FP64] - res[P.SU2_SPLIT_BF16]) <= 1e-9
