"""The D = 6144 configuration (qc64: L = N = 64, S = 0, 294 GB of FP64
operators; with their BF16 slices the resident split path would need
twice the GPU's memory) on the split path with out-of-core operators: about 200 GB of operator blocks on the device, the rest in pinned
host memory streamed per term chunk.  Sampled output blocks against the
oracle (computed block by block from its lazily generated synthetic
environment) and the symmetry of the projected Hamiltonian, at full size."""
import numpy as np
import pytest

import synth
from oracle import env as oenv
from oracle import heff as oheff
from oracle import model as omodel
from oracle import sectors as osec

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")


def test_qc64_out_of_core_sampled_blocks_and_symmetry():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if total < 250e9:
        pytest.skip("needs a GPU with at least 250 GB of memory")
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    ctx = P.Context(0, stream=torch.cuda.current_stream())
    cfg = synth.CONFIGS["qc64"]
    sec, env = workload.build(ctx, cfg, prepare_split=True, resident_bytes=int(200e9))
    info = env.info
    # the resident split path would hold the FP64 operators and their five
    # BF16 slices (10 bytes per element beside 8): 2.25 x 294 GB
    assert 2.25 * info["env_bytes"] > 2 * total
    assert info["streamed_bytes"] >= info["env_bytes"] - 200e9 - 1e9
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
    env.close()
    # <phi|H psi> = <H phi|psi>
    assert abs(phi @ Hpsi - Hphi @ psi) <= 1e-10 * np.linalg.norm(Hpsi) * np.linalg.norm(phi)
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    assert n == sec.psi_len
    order = sorted(range(len(blocks)), key=lambda f: -blocks[f].rows * blocks[f].cols)
    rng = np.random.default_rng(64)
    # a block of the largest tenth (783 x 529, 12,444 tasks, 8.7 TFLOP in the
    # oracle; the largest, 1525 x 1525, would take 37 TFLOP of CPU work), a
    # median block, the smallest (ragged) one and one from the lower half
    sel = {order[len(order) // 10], order[len(order) // 2], order[-1],
           order[int(rng.integers(len(order) // 2, len(order)))]}
    tab = omodel.qc_skeleton_table(cfg.n_left, cfg.n_right)
    e = oenv.LazySyntheticEnv(tab, cfg, left, right)
    tasks = oheff.build_tasks(tab, left, right, blocks, cfg.twoS, only_f=sel)
    F = oheff.apply_heff(tab, e, tasks, blocks, n, psi)
    idx = np.concatenate([np.arange(blocks[f].offset, blocks[f].offset + blocks[f].rows * blocks[f].cols)
                          for f in sorted(sel)])
    ref = F[idx]
    assert np.linalg.norm(Hpsi[idx] - ref) <= 1e-10 * np.linalg.norm(ref)
