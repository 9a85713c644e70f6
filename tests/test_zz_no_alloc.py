"""su2_apply_heff_static_scratch: the H.psi variant for callers that cannot
allocate device memory while they run (a pool or arena that owns the GPU, a
real-time loop).  It must give the same F as su2_apply_heff (FP64) on two
calls in a row, through the C-ABI.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_scratch_matches_apply_heff_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    ctx = P.Context(0, stream=torch.cuda.current_stream())
    cfg = synth.CONFIGS["qc16"]
    # chunks whose T fits the 64 MiB static array
    sec, env = workload.build(ctx, cfg, t_budget_bytes=48 << 20)
    assert env.info["n_chunks"] > 1
    for seed in (1, 2):
        psi = torch.from_numpy(synth.gaussian_psi(sec.psi_len, seed)).cuda()
        ref = torch.empty_like(psi)
        out = torch.full_like(psi, np.nan)
        P.apply_heff(ctx, env, psi, ref, P.SU2_FP64)
        P.apply_heff_static_scratch(ctx, env, psi, out)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_static_scratch_rejects_large_chunks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    ctx = P.Context(0, stream=torch.cuda.current_stream())
    sec, env = workload.build(ctx, synth.CONFIGS["qc16"], t_budget_bytes=1 << 30)
    # the largest term chunk's T is known to exceed the 64 MiB array
    assert env.info["t_chunk_bytes"] > 64 << 20
    x = torch.zeros(sec.psi_len, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(P.Su2Error) as ei:
        P.apply_heff_static_scratch(ctx, env, x, y)
    assert ei.value.code == P._lib.SU2_EINVAL
    assert "static scratch" in str(ei.value)
