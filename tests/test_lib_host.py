"""Host-side checks of the library (no GPU): exported symbols, sector and
task tables bit-exact against the oracle, operator blocks and the sector-
value table against the oracle, argument validation."""
import math
import os
import re

import numpy as np
import pytest

import synth
from oracle import env as oenv
from oracle import heff as oheff
from oracle import model as omodel
from oracle import sectors as osec
from paper_2309_16724_gb300 import _lib as L
from paper_2309_16724_gb300 import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "su2dmrg.h")).read()
    return sorted(set(re.findall(r"\b(su2_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    names = header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(L.SYMBOLS)


@pytest.fixture(scope="module")
def hctx():
    return L.Context(-1)


def oracle_tables(cfg, table=None, left=None, right=None):
    if left is None:
        left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    if table is None:
        table = (omodel.heisenberg_table() if cfg.site_kind == synth.SPIN_HALF
                 else omodel.qc_skeleton_table(cfg.n_left, cfg.n_right))
    tasks = oheff.build_tasks(table, left, right, blocks, cfg.twoS)
    return left, right, blocks, n, table, tasks


def task_rows(tasks):
    rows = np.zeros((len(tasks), 8), dtype=np.int32)
    v = np.zeros(len(tasks))
    for i, t in enumerate(tasks):
        ao, ai = t.A if t.A is not None else (-1, -1)
        bo, bi = t.D if t.D is not None else (-1, -1)
        rows[i] = (t.f, t.term, t.e, ao, ai, bo, bi, (1 if t.A is None else 0) | (2 if t.D is None else 0))
        v[i] = t.v
    return rows, v


CASES = [
    synth.CONFIGS["heis12"],
    synth.Config("heis10S1", synth.SPIN_HALF, 10, 10, 2, 6, 77),
    synth.Config("qc8", synth.SPATIAL_ORBITAL, 8, 8, 0, 12, 5),
    synth.Config("qc8S1", synth.SPATIAL_ORBITAL, 8, 7, 1, 10, 6),
    synth.Config("qc10S3", synth.SPATIAL_ORBITAL, 10, 9, 3, 14, 8),
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_sectors_and_tasks_bit_exact(hctx, cfg):
    left, right, blocks, n, table, tasks = oracle_tables(cfg)
    sec, env = workload.build(hctx, cfg)
    assert sec.psi_len == n
    assert sec.blocks == [(b.a, b.s1, b.s2, b.b, b.jL1, b.j2R, b.rows, b.cols, b.offset) for b in blocks]
    rows, v = env.tasks()
    orows, ov = task_rows(tasks)
    assert rows.shape == orows.shape
    assert np.array_equal(rows, orows)
    assert np.allclose(v, ov, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("which,model", [("S2", L.SU2_MODEL_CASIMIR_S2), ("N", L.SU2_MODEL_CASIMIR_N)])
def test_casimir_tables_bit_exact(hctx, which, model):
    cfg = synth.Config("c", synth.SPATIAL_ORBITAL, 8, 7, 3, 10, 3)
    table = omodel.casimir_table(cfg.site_kind, which)
    left, right, blocks, n, table, tasks = oracle_tables(cfg, table)
    sec, env = workload.build(hctx, cfg, model=model)
    rows, v = env.tasks()
    orows, ov = task_rows(tasks)
    assert np.array_equal(rows, orows)
    assert np.allclose(v, ov, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_operator_blocks_match_oracle(hctx, cfg):
    left, right, blocks, n, table, tasks = oracle_tables(cfg)
    e = oenv.build_env(table, cfg, left, right)
    sec, env = workload.build(hctx, cfg)
    checked = 0
    for (side, oid), blk in e.items():
        for (qo, qi), M in blk.items():
            got = env.operator_block(0 if side == "L" else 1, oid, qo, qi, M.shape[0], M.shape[1])
            scale = max(1.0, np.abs(M).max())
            assert np.abs(got - M).max() <= 1e-12 * scale, (side, oid, qo, qi)
            checked += 1
    assert checked > 0


def test_synthetic_entries_bit_identical(hctx):
    """Counter-generated entries are integers scaled by exact operations."""
    cfg = synth.Config("qc8", synth.SPATIAL_ORBITAL, 8, 8, 0, 12, 5)
    left, right, blocks, n, table, tasks = oracle_tables(cfg)
    e = oenv.build_env(table, cfg, left, right)
    sec, env = workload.build(hctx, cfg)
    for (side, oid), blk in e.items():
        if table.left_ops[oid].kind != omodel.RANDOM if side == "L" else table.right_ops[oid].kind != omodel.RANDOM:
            continue
        for (qo, qi), M in blk.items():
            got = env.operator_block(0 if side == "L" else 1, oid, qo, qi, M.shape[0], M.shape[1])
            assert np.array_equal(got, M)


def test_invalid_arguments(hctx):
    with pytest.raises(L.Su2Error) as ei:
        L.Sectors(hctx, [(2, 0, 1), (1, 1, 1)], [(1, 1, 1)], synth.SPATIAL_ORBITAL, 4, 0)
    assert ei.value.code == L.SU2_EINVAL
    with pytest.raises(L.Su2Error):
        L.Sectors(hctx, [(1, 1, 0)], [(1, 1, 1)], synth.SPATIAL_ORBITAL, 4, 0)
    cfg = synth.CONFIGS["heis12"]
    lch, rch = workload.chains(cfg)
    sec = L.Sectors(hctx, lch[-1], rch[-1], cfg.site_kind, cfg.N, cfg.twoS)
    with pytest.raises(L.Su2Error):
        L.Environment(hctx, sec, 9, lch, rch)
    with pytest.raises(L.Su2Error):   # chain end differs from the sectors
        L.Environment(hctx, sec, L.SU2_MODEL_HEISENBERG, lch[:-1], rch)
    with pytest.raises(L.Su2Error):   # device work on a host-only context
        env = L.Environment(hctx, sec, L.SU2_MODEL_HEISENBERG, lch, rch, seed=1)
        L.apply_heff(hctx, env, 8, 4096)


def test_flop_count_matches_oracle_dedup(hctx):
    cfg = synth.Config("qc8", synth.SPATIAL_ORBITAL, 8, 8, 0, 12, 5)
    left, right, blocks, n, table, tasks = oracle_tables(cfg)
    k1 = {}
    k2 = 0
    for t in tasks:
        E, F = blocks[t.e], blocks[t.f]
        if t.D is not None:
            k1[(table.terms[t.term].D, t.D, t.e)] = 2 * E.rows * E.cols * F.cols
        if t.A is not None:
            k2 += 2 * F.rows * E.rows * F.cols
    sec, env = workload.build(hctx, cfg)
    assert env.info["flops_su2"] == sum(k1.values()) + k2
    D = sum(d for (_, _, d) in left)
    Deff = sum(d * (s + 1) for (_, s, d) in left)
    assert env.info["r_d"] == pytest.approx(Deff / D)


def test_shard_options(hctx):
    """A shard rank outside [0, count) is rejected; the shards of a count
    partition the task list (each task in exactly one shard)."""
    cfg = synth.Config("qc8", synth.SPATIAL_ORBITAL, 8, 8, 0, 12, 5)
    lch, rch = workload.chains(cfg)
    sec = L.Sectors(hctx, lch[-1], rch[-1], cfg.site_kind, cfg.N, cfg.twoS)
    kw = dict(n_left=cfg.n_left, n_right=cfg.n_right, seed=cfg.seed)
    with pytest.raises(L.Su2Error) as ei:
        L.Environment(hctx, sec, L.SU2_MODEL_QC_SKELETON, lch, rch, shard=(3, 3), **kw)
    assert ei.value.code == L.SU2_EINVAL
    full = L.Environment(hctx, sec, L.SU2_MODEL_QC_SKELETON, lch, rch, **kw)
    rows, v = full.tasks()
    key = lambda r: tuple(int(x) for x in r[:7])
    want = sorted(key(r) for r in rows)
    got = []
    for r in range(3):
        part = L.Environment(hctx, sec, L.SU2_MODEL_QC_SKELETON, lch, rch, shard=(r, 3), **kw)
        prow, _ = part.tasks()
        assert len(prow) > 0
        got += [key(x) for x in prow]
    assert sorted(got) == want


def test_sweep_needs_a_device_context(hctx):
    """su2_sweep_create on a host-only context returns SU2_EINVAL with its
    reason (the sweep's Davidson runs on the GPU; there is no host path)."""
    cfg = synth.CONFIGS["heis12"]
    chain = synth.bond_sector_chain(cfg, cfg.L - 2)
    with pytest.raises(L.Su2Error) as ei:
        L.Sweep(hctx, None, None, chain, cfg.N, cfg.D)
    assert ei.value.code == L.SU2_EINVAL and "device context" in str(ei.value)
