"""Failure detection on the GPU without faulting it.

* A bounded device wait that runs out: the split GEMM's work-loop waits are
  given a limit of a few polls (su2_env_opts.spin_limit), so its CTAs give up
  almost at once.  The kernel sets the device status word and returns (each
  CTA still waits the full limit for its own copies and MMAs); the host reads
  SU2_ETIMEOUT, and the same context then computes a correct H.psi with an
  environment built with the normal limit.
* The host watchdog (su2_ctx_wait): a queue of FP64 H.psi is still running
  after a 1 ms limit (SU2_ETIMEOUT, nothing is killed) and finishes under a
  generous one.
* The binding rejects buffers of the wrong dtype, length, layout or device
  before the library is called.
"""
import numpy as np
import pytest

import synth

from gpu_common import oracle_apply, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    torch.cuda.init()
    return P.Context(0, stream=torch.cuda.current_stream())


def test_split_wait_runs_out_and_context_recovers(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc16"]
    assert ctx.status() == 0
    sec, env_short = workload.build(ctx, cfg, prepare_split=True, n_slices=5, spin_limit=2)
    psi = synth.gaussian_psi(sec.psi_len, 3)
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    P.apply_heff(ctx, env_short, x, y, P.SU2_SPLIT_BF16)
    assert ctx.status() == P._lib.SU2_ETIMEOUT
    assert ctx.status() == 0                     # read and cleared
    # a synchronising call reports the timeout as its return code
    out_h = np.empty(sec.psi_len)
    with pytest.raises(P.Su2Error) as ei:
        P.apply_heff_host(ctx, env_short, psi, out_h, P.SU2_SPLIT_BF16)
    assert ei.value.code == P._lib.SU2_ETIMEOUT
    env_short.close()
    # the context is still usable: a normal environment gives the right F
    sec2, env = workload.build(ctx, cfg, prepare_split=True, n_slices=5)
    P.apply_heff(ctx, env, x, y, P.SU2_SPLIT_BF16)
    assert ctx.status() == 0
    ref = oracle_apply(oracle_problem(cfg), psi)
    assert rel_err(y.cpu().numpy(), ref) <= 1e-10


def test_davidson_step_reports_timeout(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc16"]
    sec, env = workload.build(ctx, cfg, prepare_split=True, n_slices=5, spin_limit=2)
    psi0 = torch.from_numpy(synth.gaussian_psi(sec.psi_len, 4)).cuda()
    dav = P.Davidson(ctx, env, psi0, tol=1e-8, prec=P.SU2_SPLIT_BF16)
    with pytest.raises(P.Su2Error) as ei:
        dav.step()
    assert ei.value.code == P._lib.SU2_ETIMEOUT
    dav.close()
    assert ctx.status() == 0


def test_host_watchdog(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc16"]
    sec, env = workload.build(ctx, cfg)
    x = torch.from_numpy(synth.gaussian_psi(sec.psi_len, 5)).cuda()
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    for _ in range(30):                          # ~0.2 s of FP64 work each
        P.apply_heff(ctx, env, x, y, P.SU2_FP64)
    assert ctx.wait(0.001) == P._lib.SU2_ETIMEOUT
    assert ctx.wait(600.0) == P._lib.SU2_OK
    assert ctx.wait(0.0) == P._lib.SU2_OK        # idle stream


def test_binding_rejects_bad_buffers(ctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.CONFIGS["qc16"]
    sec, env = workload.build(ctx, cfg)
    n = sec.psi_len
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    bad_cases = [
        torch.zeros(n, dtype=torch.float32, device="cuda"),         # dtype
        torch.zeros(n - 1, dtype=torch.float64, device="cuda"),     # too short
        torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2],  # strided
        torch.zeros(n, dtype=torch.float64),                        # host tensor for a device entry
        np.zeros(n),                                                # numpy for a device entry
    ]
    for b in bad_cases:
        with pytest.raises(P.Su2Error) as ei:
            P.apply_heff(ctx, env, b, good)
        assert ei.value.code == P._lib.SU2_EINVAL
        with pytest.raises(P.Su2Error) as ei:
            P.apply_heff(ctx, env, good, b)
        assert ei.value.code == P._lib.SU2_EINVAL
    with pytest.raises(P.Su2Error) as ei:                           # device tensor for a host entry
        P.apply_heff_host(ctx, env, good, np.zeros(n))
    assert ei.value.code == P._lib.SU2_EINVAL
    with pytest.raises(P.Su2Error):
        P.apply_heff_host(ctx, env, np.zeros(n, dtype=np.float32), np.zeros(n))
