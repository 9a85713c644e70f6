"""Flop bookkeeping of the metric (SU(2) and U(1)-equivalent flops).

* The paper's Table 1 ratios follow from its own columns with the readings
  R_D = D_U(1)^eff / D and R_CC = CC_U(1) / CC_SU(2) (golden fixture with
  the printed values).
* R_D of the library is sum_q d_q (2S_q + 1) / sum_q d_q of the left bond.
* The U(1)-expanded count has a closed form when every bond sector is a
  singlet and the sites are spin-1/2: each SU(2) two-site block (a, b) of
  total spin 0 becomes the two U(1) blocks (up, dn) and (dn, up) of the same
  size, so the count is exactly twice the SU(2) count (R_CC = 2, R_D = 1).
* On the ab initio workloads R_CC exceeds R_D, as in Table 1.
"""
import os

import numpy as np
import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table1_ratios_follow_from_its_columns():
    rows = [list(map(float, l.split())) for l in open(os.path.join(HERE, "golden", "table1_ratios.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for D, Deff, RD, ccu1, ccsu2, RCC in rows:
        assert round(Deff / D, 2) == RD
        assert round(ccu1 / ccsu2, 2) == RCC
    # both ratios grow with D up to 4096 in the table; R_CC exceeds R_D from D = 2048 on
    assert rows[1][5] > rows[1][2] and rows[2][5] > rows[2][2]


@pytest.fixture(scope="module")
def hctx():
    import paper_2309_16724_gb300 as P
    return P.Context(-1)


def test_r_d_is_the_multiplet_weighted_dimension(hctx):
    from paper_2309_16724_gb300 import workload
    for name in ("heis12", "qc16"):
        cfg = synth.CONFIGS[name]
        sec, env = workload.build(hctx, cfg)
        left = sec.left
        want = sum(d * (S + 1) for (_, S, d) in left) / sum(d for (_, _, d) in left)
        assert abs(env.info["r_d"] - want) < 1e-15
        assert abs(env.info["flops_u1_equiv"] - env.info["flops_su2"] * want) <= 1e-12 * env.info["flops_u1_equiv"]


def test_u1_count_closed_form_for_singlet_bonds(hctx):
    import paper_2309_16724_gb300 as P
    left_chain = [[(0, 0, 1)], [(4, 0, 3)]]
    right_chain = [[(0, 0, 1)], [(4, 0, 2)]]
    sec = P.Sectors(hctx, left_chain[-1], right_chain[-1], synth.SPIN_HALF, 10, 0)
    env = P.Environment(hctx, sec, P.SU2_MODEL_CASIMIR_N, left_chain, right_chain, n_left=1, n_right=1)
    i = env.info
    # SU(2): one 3 x 2 block; N_L: A T = 2*3*3*2, N_R: E D^T = 2*3*2*2
    assert i["flops_su2"] == 2 * 3 * 3 * 2 + 2 * 3 * 2 * 2
    assert i["flops_u1_counted"] == 2 * i["flops_su2"]
    assert i["r_cc"] == 2.0 and i["r_d"] == 1.0


def test_u1_ratio_exceeds_r_d_on_ab_initio(hctx):
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    cfg = synth.Config("ab12", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 1002)
    sec, env = workload.build(hctx, cfg, model=P.SU2_MODEL_AB_INITIO)
    i = env.info
    assert 1.0 < i["r_d"] < i["r_cc"]
