"""Term sharding of H.psi (the multi-GPU partition, one shard per rank).

CPU: two gloo ranks each build their shard of the environment through the
C-ABI (host context), take its terms, compute their partial F with the
oracle and all-reduce it; the sum must equal the full oracle H.psi and the
term sets must partition the terms.  GPU: two shards built on one device
sum to the full H.psi (FP64 and split paths).
"""
import os
import socket

import numpy as np
import pytest

import synth
from gpu_common import oracle_problem, rel_err
from oracle import heff as oheff

CFG = synth.Config("qc10S3", synth.SPATIAL_ORBITAL, 10, 9, 3, 40, 8)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2309_16724_gb300 as P
        from paper_2309_16724_gb300 import workload
        ctx = P.Context(-1)
        sec, env = workload.build(ctx, CFG, shard=(rank, world))
        rows, _ = env.tasks()
        terms = set(int(t) for t in rows[:, 1])
        p = oracle_problem(CFG)
        mine = [t for t in p["tasks"] if t.term in terms]
        psi = synth.gaussian_psi(p["n"], 3)
        F = torch.from_numpy(oheff.apply_heff(p["table"], p["env"], mine, p["blocks"], p["n"], psi))
        dist.all_reduce(F)  # sum over the shards
        allt = [None] * world
        dist.all_gather_object(allt, sorted(terms))
        if rank == 0:
            full = oheff.apply_heff(p["table"], p["env"], p["tasks"], p["blocks"], p["n"], psi)
            q.put((rel_err(F.numpy(), full), allt, len(mine), len(p["tasks"]), sorted({t.term for t in p["tasks"]})))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_term_shards_sum_to_full_hpsi_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs)
    err, allt, n0, ntot, terms = q.get()
    assert err <= 1e-13, err
    a, b = set(allt[0]), set(allt[1])
    assert not (a & b)
    assert sorted(a | b) == terms
    assert 0 < n0 < ntot


@pytest.mark.gpu
def test_term_shards_sum_on_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload
    ctx = P.Context(0, stream=torch.cuda.current_stream())
    cfg = synth.Config("qc12D100", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 9)
    sec, full = workload.build(ctx, cfg, prepare_split=True)
    shards = [workload.build(ctx, cfg, prepare_split=True, shard=(r, 2))[1] for r in range(2)]
    x = torch.from_numpy(synth.gaussian_psi(sec.psi_len, 2)).cuda()
    for prec, tol in ((P.SU2_FP64, 1e-13), (P.SU2_SPLIT_BF16, 1e-10)):
        y = torch.empty_like(x)
        P.apply_heff(ctx, full, x, y, prec)
        s = torch.zeros_like(x)
        for env in shards:
            z = torch.empty_like(x)
            P.apply_heff(ctx, env, x, z, prec)
            s += z
        assert ctx.status() == 0
        assert rel_err(s.cpu().numpy(), y.cpu().numpy()) <= tol
    assert sum(e.info["n_tasks"] for e in shards) == full.info["n_tasks"]
