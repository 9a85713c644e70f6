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


def test_hash_group_order_reaches_every_group():
    """Fig. 2 (Sec. III.D): group_count consecutive picks of a worker visit
    every group once, whatever gcd(group_count, workers); workers start on
    different groups; without the cycle shift a worker would miss groups when
    the counts share a factor (brute force over small counts)."""
    import paper_2309_16724_gb300 as P
    for G in range(1, 31):
        for W in range(1, 13):
            starts = set()
            for w in range(W):
                seq = [P.hash_group(w, W, G, i) for i in range(G)]
                assert sorted(seq) == list(range(G)), (G, W, w, seq)
                starts.add(seq[0])
            assert len(starts) == min(W, G)
    # 6 groups, 2 workers: steps of 2 alone would stay in the even groups
    assert [P.hash_group(0, 2, 6, i) for i in range(6)] == [0, 2, 4, 1, 3, 5]
    assert [P.hash_group(1, 2, 6, i) for i in range(6)] == [1, 3, 5, 2, 4, 0]
    assert sorted({(2 * i) % 6 for i in range(6)}) != list(range(6))
    with pytest.raises(P.Su2Error):
        P.hash_group(2, 2, 6, 0)


BATCH = 256


def _book_rank(rank, world, port, q):
    import datetime
    import torch
    import torch.distributed as dist
    # the process group's own key-value store doubles as the Contract Book
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=datetime.timedelta(seconds=120))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world)
    try:
        import paper_2309_16724_gb300 as P
        p = oracle_problem(CFG)
        groups = {}
        for t in p["tasks"]:                     # a group: the tasks into one output block
            groups.setdefault(t.f, []).append(t)
        keys = sorted(groups)
        G = len(keys)
        mine = []
        dist.barrier()                           # start claiming together
        for i in range(G):                       # the worker's hashed group order
            g = keys[P.hash_group(rank, world, G, i)]
            while True:                          # claim the group's tasks from the shared book, a batch at a time
                end = store.add(f"group{g}", BATCH)
                if end - BATCH >= len(groups[g]):
                    break
                mine.extend(groups[g][end - BATCH:end])
        psi = synth.gaussian_psi(p["n"], 3)
        F = torch.from_numpy(oheff.apply_heff(p["table"], p["env"], mine, p["blocks"], p["n"], psi))
        dist.all_reduce(F)
        counts = [None] * world
        dist.all_gather_object(counts, [(t.f, t.term, t.e) for t in mine])
        if rank == 0:
            full = oheff.apply_heff(p["table"], p["env"], p["tasks"], p["blocks"], p["n"], psi)
            flat = [c for per in counts for c in per]
            q.put((rel_err(F.numpy(), full), len(flat), len(set(flat)), [len(per) for per in counts],
                   len(p["tasks"])))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_contract_book_claims_in_hash_order_gloo():
    """Three CPU ranks claim tasks group by group in the Fig. 2 order from a
    shared counter per group; every task is claimed once and the partial F
    sum to H.psi."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_book_rank, args=(r, 3, port, q)) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
    assert all(p.exitcode == 0 for p in procs)
    err, nclaimed, nunique, per_rank, ntot = q.get()
    assert err <= 1e-13, err
    assert nclaimed == nunique == ntot
    assert sum(per_rank) == ntot


def _gpu_rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2309_16724_gb300 as P
        from paper_2309_16724_gb300 import workload
        torch.cuda.set_device(0)
        ctx = P.Context(0, stream=torch.cuda.current_stream())
        cfg = synth.Config("qc12D100", synth.SPATIAL_ORBITAL, 12, 12, 0, 100, 9)
        sec, env = workload.build(ctx, cfg, prepare_split=True, shard=(rank, world))
        x = torch.from_numpy(synth.gaussian_psi(sec.psi_len, 2)).cuda()
        out = {}
        for prec in (P.SU2_FP64, P.SU2_SPLIT_BF16):
            y = torch.empty_like(x)
            P.apply_heff(ctx, env, x, y, prec)
            torch.cuda.synchronize()
            assert ctx.status() == 0
            F = y.cpu()
            dist.all_reduce(F)                   # the sum of the partial F (host tensors)
            out[prec] = F.numpy()
        if rank == 0:
            _, full = workload.build(ctx, cfg, prepare_split=True)
            ref = {}
            for prec in (P.SU2_FP64, P.SU2_SPLIT_BF16):
                y = torch.empty_like(x)
                P.apply_heff(ctx, full, x, y, prec)
                torch.cuda.synchronize()
                ref[prec] = y.cpu().numpy()
            q.put([rel_err(out[p_], ref[p_]) for p_ in (P.SU2_FP64, P.SU2_SPLIT_BF16)])
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_two_rank_term_shards_through_the_library():
    """Two processes (ranks of a gloo group) each apply their term shard with
    the library's kernels on the one GPU (independent launches, nothing
    waits on the other rank) and sum the partial F on the host: equal to the
    single-process H.psi (FP64 1e-13, split 1e-10)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_gpu_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=900)
    assert all(p.exitcode == 0 for p in procs)
    e64, esp = q.get()
    assert e64 <= 1e-13 and esp <= 1e-10, (e64, esp)
