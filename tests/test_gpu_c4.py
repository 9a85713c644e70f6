"""The D = 4096 configuration (qc48: L = N = 48, S = 0) on the split path:
sampled output blocks (the largest among them) against the oracle (computed block by block from its
lazily generated synthetic environment) and the symmetry of the projected
Hamiltonian, at full size."""
import numpy as np
import pytest

import synth
from oracle import env as oenv
from oracle import heff as oheff
from oracle import model as omodel
from oracle import sectors as osec

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


def test_qc48_split_sampled_blocks_and_symmetry():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    ctx = P.Context(0, stream=torch.cuda.current_stream())
    cfg = synth.CONFIGS["qc48"]
    sec, env = workload.build(ctx, cfg, prepare_split=True)
    psi = synth.gaussian_psi(sec.psi_len, synth.psi_seed(cfg))
    phi = synth.gaussian_psi(sec.psi_len, 98)
    x = torch.from_numpy(psi).cuda()
    u = torch.from_numpy(phi).cuda()
    y = torch.empty_like(x)
    v = torch.empty_like(x)
    P.apply_heff(ctx, env, x, y, P.SU2_SPLIT_BF16)
    P.apply_heff(ctx, env, u, v, P.SU2_SPLIT_BF16)
    assert ctx.status() == 0
    Hpsi, Hphi = y.cpu().numpy(), v.cpu().numpy()
    # <phi|H psi> = <H phi|psi>
    assert abs(phi @ Hpsi - Hphi @ psi) <= 1e-10 * np.linalg.norm(Hpsi) * np.linalg.norm(phi)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    assert n == sec.psi_len
    order = sorted(range(len(blocks)), key=lambda f: -blocks[f].rows * blocks[f].cols)
    rng = np.random.default_rng(48)
    # the largest block (1017 x 1017, 3649 tasks, 6.3 TFLOP in the oracle), a
    # median block, the smallest (ragged) one and one from the lower half
    sel = {order[0], order[len(order) // 2], order[-1], order[int(rng.integers(len(order) // 2, len(order)))]}
    tab = omodel.qc_skeleton_table(cfg.n_left, cfg.n_right)
    e = oenv.LazySyntheticEnv(tab, cfg, left, right)
    tasks = oheff.build_tasks(tab, left, right, blocks, cfg.twoS, only_f=sel)
    F = oheff.apply_heff(tab, e, tasks, blocks, n, psi)
    idx = np.concatenate([np.arange(blocks[f].offset, blocks[f].offset + blocks[f].rows * blocks[f].cols)
                          for f in sorted(sel)])
    ref = F[idx]
    assert np.linalg.norm(Hpsi[idx] - ref) <= 1e-10 * np.linalg.norm(ref)
