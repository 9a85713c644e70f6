"""The out-of-core plan (Sec. III.E-F) on the host.

A host context makes the plan of an environment built with a device budget
(chunk boundaries, which blocks stay on the device, the logical layout of
the arenas) and lays its host arenas out that way.  Checked: every operator
block reads back equal to the resident environment's, the task table and
the resulting H_eff are unchanged, the plan's byte counts add up, and a
larger budget keeps more blocks resident.
"""
import numpy as np
import pytest

import synth

from test_lib_abinitio import lib_apply

L_ = pytest.importorskip("paper_2309_16724_gb300._lib")

MB = 1 << 20


@pytest.fixture(scope="module")
def hctx():
    import paper_2309_16724_gb300 as P
    return P.Context(-1)


def blocks_of(env, sec):
    import paper_2309_16724_gb300 as P
    ad, dd, _, _ = env.terms()
    out = {}
    for side, S in ((0, sec.left), (1, sec.right)):
        for op in sorted(set((ad if side == 0 else dd).tolist()) - {0}):
            for qo in range(len(S)):
                for qi in range(len(S)):
                    try:
                        out[(side, op, qo, qi)] = env.operator_block(side, op, qo, qi, S[qo][2], S[qi][2])
                    except P.Su2Error:
                        pass
    return out


@pytest.mark.parametrize("name,model", [("qc12D100", "skeleton"), ("ab10", "ab_initio")])
def test_out_of_core_plan_keeps_every_block(hctx, name, model):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    if name == "qc12D100":
        cfg = synth.Config("qc12D100", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 9)
    else:
        cfg = synth.Config("ab10", synth.SPATIAL_ORBITAL, 10, 10, 0, 60, 1002)
    m = P.SU2_MODEL_AB_INITIO if model == "ab_initio" else P.SU2_MODEL_QC_SKELETON
    sec, env_in = workload.build(hctx, cfg, model=m)
    _, env_oc = workload.build(hctx, cfg, model=m, t_budget_bytes=MB // 4, resident_bytes=1)
    info = env_oc.info
    assert info["n_io_chunks"] >= 3
    assert info["streamed_bytes"] > 0
    assert info["resident_bytes"] + info["streamed_bytes"] >= info["env_bytes"]
    assert env_in.info["n_io_chunks"] == 0 and env_in.info["streamed_bytes"] == 0
    a, b = blocks_of(env_in, sec), blocks_of(env_oc, sec)
    assert a.keys() == b.keys() and len(a) > 50
    for k in a:
        assert np.array_equal(a[k], b[k])
    r1, v1 = env_in.tasks()
    r2, v2 = env_oc.tasks()
    assert np.array_equal(r1, r2) and np.array_equal(v1, v2)
    psi = synth.gaussian_psi(sec.psi_len, 3)
    F1, F2 = lib_apply(env_in, sec)(psi), lib_apply(env_oc, sec)(psi)
    assert np.array_equal(F1, F2)
    # a budget as large as the operators keeps every block on the device
    _, env_all = workload.build(hctx, cfg, model=m, t_budget_bytes=MB // 4,
                                resident_bytes=int(2 * info["env_bytes"]) + MB)
    assert env_all.info["streamed_bytes"] == 0
    _, env_half = workload.build(hctx, cfg, model=m, t_budget_bytes=MB // 4,
                                 resident_bytes=int(info["resident_bytes"] + info["streamed_bytes"] // 2))
    assert 0 < env_half.info["streamed_bytes"] < info["streamed_bytes"]
    for e in (env_in, env_oc, env_all, env_half):
        e.close()
