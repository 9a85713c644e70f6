"""GPU parity of the split-precision (BF16 slices on tcgen05) path.

Bar: relative 2-norm error of H.psi <= 1e-10 against the FP64
oracle and against the GPU FP64 path on the same inputs; the device status
word stays clear (no bounded wait gave up).
"""
import numpy as np
import pytest

import synth

from gpu_common import oracle_apply, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_SPLIT = 1e-10


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    return P.Context(0, stream=torch.cuda.current_stream())


def run(ctx, env, psi, prec):
    import paper_2309_16724_gb300 as P
    x = torch.from_numpy(psi).cuda()
    y = torch.empty_like(x)
    P.apply_heff(ctx, env, x, y, prec)
    assert ctx.status() == 0
    return y.cpu().numpy()


CASES = [
    synth.Config("qc8", synth.SPATIAL_ORBITAL, 8, 8, 0, 12, 5),
    synth.Config("qc10S3", synth.SPATIAL_ORBITAL, 10, 9, 3, 40, 8),
    synth.Config("qc12D100", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 9),
    synth.CONFIGS["heis12"],
    synth.CONFIGS["qc16"],
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_split_matches_oracle(ctx, cfg):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    p = oracle_problem(cfg)
    psi = synth.gaussian_psi(p["n"], synth.psi_seed(cfg))
    F = oracle_apply(p, psi)
    sec, env = workload.build(ctx, cfg, prepare_split=True)
    G = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    assert rel_err(G, F) <= TOL_SPLIT, rel_err(G, F)
    H = run(ctx, env, psi, P.SU2_FP64)
    assert rel_err(G, H) <= TOL_SPLIT


def test_split_chunking_and_repeat(ctx):
    """Many term chunks, and two calls in a row give identical results."""
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = CASES[2]
    sec, env = workload.build(ctx, cfg, prepare_split=True, t_budget_bytes=1 << 20)
    psi = synth.gaussian_psi(sec.psi_len, 4)
    a = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    b = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    assert np.array_equal(a, b)
    H = run(ctx, env, psi, P.SU2_FP64)
    assert rel_err(a, H) <= TOL_SPLIT


@pytest.mark.parametrize("S,tol", [(3, 1e-5), (4, 1e-7), (5, 1e-10), (6, 1e-11)])
def test_slice_count_controls_error(ctx, S, tol):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = CASES[2]
    sec, env = workload.build(ctx, cfg, prepare_split=True, n_slices=S)
    psi = synth.gaussian_psi(sec.psi_len, 6)
    G = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    H = run(ctx, env, psi, P.SU2_FP64)
    assert rel_err(G, H) <= tol


@pytest.mark.parametrize("tol", [1e-5, 3e-11, 1e-14])
def test_autotune_picks_slices_and_stage_depth(ctx, tol):
    """The autotuner's slice count is the smallest whose H.psi differs from the
    six-slice one by <= tol; the prepared path then meets that bound against
    the FP64 path (up to the six-slice error itself), and its stage depth is a
    valid one."""
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = CASES[2]
    sec, env = workload.build(ctx, cfg, autotune=True, split_tol=tol)
    S, sk, est = env.info["split_slices"], env.info["split_stage_k"], env.info["split_err_est"]
    assert 2 <= S <= 6 and sk in (1, 2, 3, 4, 6)
    if S < 6:
        assert 0.0 <= est <= tol
    else:
        assert est == -1.0
    if tol >= 1e-5:
        assert S <= 4
    if tol <= 1e-14:
        assert S == 6
    psi = synth.gaussian_psi(sec.psi_len, 6)
    G = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    H = run(ctx, env, psi, P.SU2_FP64)
    assert rel_err(G, H) <= max(10 * tol, 1e-11)


def test_degenerate_inputs(ctx):
    """psi = 0 gives F = 0 exactly on both paths (zero rows and columns take
    the sentinel exponents); psi non-zero in one block only still matches the
    oracle."""
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = CASES[2]
    p = oracle_problem(cfg)
    sec, env = workload.build(ctx, cfg, prepare_split=True)
    z = np.zeros(sec.psi_len)
    for prec in (P.SU2_FP64, P.SU2_SPLIT_BF16):
        assert not np.any(run(ctx, env, z, prec))
    blk = max(p["blocks"], key=lambda b: b.rows * b.cols)
    one = np.zeros(p["n"])
    one[blk.offset:blk.offset + blk.rows * blk.cols] = synth.gaussian_psi(blk.rows * blk.cols, 11)
    F = oracle_apply(p, one)
    assert rel_err(run(ctx, env, one, P.SU2_SPLIT_BF16), F) <= TOL_SPLIT
    assert rel_err(run(ctx, env, one, P.SU2_FP64), F) <= 1e-12


@pytest.mark.parametrize("which", ["S2", "N"])
def test_split_casimir(ctx, which):
    """Total spin squared (as a sum of S_i.S_j) and particle number through the
    whole split machinery: S(S+1) psi and N psi."""
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("c", synth.SPATIAL_ORBITAL, 12, 11, 3, 120, 4)
    model = P.SU2_MODEL_CASIMIR_S2 if which == "S2" else P.SU2_MODEL_CASIMIR_N
    sec, env = workload.build(ctx, cfg, model=model, prepare_split=True)
    psi = synth.gaussian_psi(sec.psi_len, 1)
    G = run(ctx, env, psi, P.SU2_SPLIT_BF16)
    want = 1.5 * 2.5 if which == "S2" else 11.0
    assert rel_err(G, want * psi) <= TOL_SPLIT
