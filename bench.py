"""Benchmark of the SU(2) two-site H.psi (Eq. 2) on GB300.

One step = one full H.psi (every operator-table row, every task) of the
seeded synthetic workload, inputs resident in HBM.  Prints one JSON line.
The default workload is the L = N = 48, D = 4096 ab initio configuration
(qc48).  Beside the split-precision value the line carries the native-FP64
path's rate on the same workload (a term shard of it, timed), the split/FP64
ratio and the split error against the FP64 result on that shard, and the
oracle timed on the host cores on a flop-weighted sample; besides, the ab
initio block (qc32 from the seeded integrals), the out-of-core block (qc64)
and two sweeps with wavefunction prediction (the Heisenberg chain and qc16).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME]
                  [--prec split|fp64] [--impl ours|reference]

Multi-GPU (torchrun): every rank runs an independent replica of the
workload (the path needs no exchange on one node), value = total flops of
all ranks / max time over ranks ("weak" scaling).
"""
from __future__ import annotations

import argparse
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "H·ψ TFLOPS/GB300 (SU(2), U(1)-equiv): split-prec vs FP64 at ≤1e-10 rel err"
DEFAULT_CONFIG = "qc48"   # L = N = 48, D = 4096: the batching configuration the throughput target is set on
FP64_PEAK_TFLOPS = 1.25   # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal FP64 rate)


def k2_traffic(workload, slices, stage_k):
    """DRAM bytes per K2 launch from the committed ncu capture, or None when the
    split sources changed since it was taken or the workload differs."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    src = os.path.join(root, "paper_2309_16724_gb300", "csrc")
    try:
        txt = open(os.path.join(root, "profiles", "split_gemm_dram_qc48.md")).read()
        h = hashlib.sha256()
        for f in ("split_gemm.cuh", "heff_split.cu"):
            h.update(open(os.path.join(src, f), "rb").read())
    except OSError:
        return None
    kv = dict(re.findall(r"(\w+): (\S+)", txt.split("Machine-readable", 1)[-1]))
    if kv.get("sources_sha256_16") != h.hexdigest()[:16]:
        return None
    if (kv.get("workload"), kv.get("slices"), kv.get("stage_k16")) != (workload, str(slices), str(stage_k)):
        return None
    return float(kv["k2_split_traffic_bytes_per_launch"])


def workload_config(cfg):
    """The workload as both arms name it (the same dict on the library's line
    and on the oracle's): configuration, sizes, operator source and the L2
    rule between timed steps."""
    return {"workload": cfg.name, "L": cfg.L, "N": cfg.N, "twoS": cfg.twoS, "D": cfg.D,
            "operators": "synthetic-entry environments (ab initio normal/complementary term "
                         "structure, counter-generated entries)" if cfg.site_kind else
                         "Heisenberg, renormalised from a seeded MPS",
            "l2": "flushed between steps (256 MB write)"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


_ORACLE_WORKER = r"""
import os, sys, time, json, pickle
sys.path.insert(0, ROOT)
import numpy as np, synth
from oracle import heff
w, W, path, repeats, warm = int(sys.argv[1]), int(sys.argv[2]), sys.argv[3], int(sys.argv[4]), int(sys.argv[5])
with open(path, "rb") as f:
    d = pickle.load(f)
tab, e, blocks, n, psi, parts = d["table"], d["env"], d["blocks"], d["n"], d["psi"], d["parts"]
tasks = parts[w]
print("ready", flush=True)
sys.stdin.readline()  # start together
for r in range(warm):
    heff.apply_heff(tab, e, tasks, blocks, n, psi)
times = []
for r in range(repeats):
    t0 = time.perf_counter(); heff.apply_heff(tab, e, tasks, blocks, n, psi); times.append(time.perf_counter() - t0)
print(json.dumps({"times": times}), flush=True)
"""


def _oracle_sample(cfg_name: str, W: int, frac: float = 0.02, min_flops: float = 2e10):
    """The oracle's problem for a config and a bounded sample of its H.psi:
    the full H.psi when it is small, else output blocks drawn with
    probability proportional to their flops (seeded, without replacement)
    until the drawn blocks hold `frac` of the flops (at least `min_flops`);
    every task into a drawn block is kept.  Tasks are dealt to W workers,
    longest first.  Returns (pickle path, sample flops, total flops,
    description)."""
    import pickle
    import numpy as np
    from oracle import env as oenv, heff as oheff, model as omodel, sectors as osec
    cfg = synth.CONFIGS[cfg_name]
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    tab = (omodel.heisenberg_table() if cfg.site_kind == synth.SPIN_HALF
           else omodel.qc_skeleton_table(cfg.n_left, cfg.n_right))

    def work(ts):
        k1, k2 = {}, 0
        for t in ts:
            E, F = blocks[t.e], blocks[t.f]
            if t.D is not None:
                k1[(tab.terms[t.term].D, t.D, t.e)] = 2 * E.rows * E.cols * F.cols
            if t.A is not None:
                k2 += 2 * F.rows * E.rows * F.cols
        return sum(k1.values()) + k2

    if n < 1_000_000:
        e = oenv.build_env(tab, cfg, left, right)
        sample_tasks = oheff.build_tasks(tab, left, right, blocks, cfg.twoS)
        total = work(sample_tasks)
        flops = total
        desc = f"full H.psi of {cfg_name} (all tasks) on {W} processes"
    else:
        e = oenv.LazySyntheticEnv(tab, cfg, left, right)
        all_tasks = oheff.build_tasks(tab, left, right, blocks, cfg.twoS)
        by_f = {}
        for t in all_tasks:
            by_f.setdefault(t.f, []).append(t)
        wf = {f: work(ts) for f, ts in by_f.items()}
        total = sum(wf.values())
        rng = np.random.default_rng(20230928)
        fs = sorted(wf)
        p = np.array([wf[f] for f in fs], dtype=np.float64)
        order = rng.choice(len(fs), size=len(fs), replace=False, p=p / p.sum())
        keep, acc = [], 0
        target = max(frac * total, min_flops)
        for i in order:
            if acc >= target:
                break
            keep.append(fs[i])
            acc += wf[fs[i]]
        sample_tasks = [t for f in keep for t in by_f[f]]
        flops = acc
        desc = (f"{len(keep)} of {len(blocks)} output blocks of {cfg_name} drawn with probability proportional "
                f"to their flops ({100 * flops / total:.1f} % of the H.psi flops, every task into them), "
                f"on {W} processes; rate extrapolated to the whole H.psi")

    def cost(t):
        E, F = blocks[t.e], blocks[t.f]
        return 2 * (F.rows * E.rows * E.cols + F.rows * E.cols * F.cols)

    load = [0] * W
    parts = [[] for _ in range(W)]
    for i in sorted(range(len(sample_tasks)), key=lambda i: (-cost(sample_tasks[i]), i)):
        r = min(range(W), key=lambda k: (load[k], k))
        load[r] += cost(sample_tasks[i])
        parts[r].append(sample_tasks[i])
    psi = synth.gaussian_psi(n, synth.psi_seed(cfg))
    path = tempfile.mktemp(prefix="oracle_sample_", suffix=".pkl")
    with open(path, "wb") as f:
        pickle.dump({"table": tab, "env": e, "blocks": blocks, "n": n, "psi": psi, "parts": parts}, f)
    return path, flops, total, desc


def oracle_cpu_baseline(cfg_name: str, repeats: int, workers: int = 0, warmup: int = 0):
    """Times the FP64 oracle (as it stands) on the host cores: `workers`
    processes (default: one per core), one BLAS thread each, `warmup`
    untimed repeats first, then `repeats` timed ones started together.  The
    work is the full H.psi of a small config, else a flop-weighted sample of
    output blocks (`_oracle_sample`).  Returns (TFLOP/s, cores, sample
    description, seconds per repeat): the sample's flops over the slowest
    worker's time, median over the repeats.  Flops follow the library's
    definition (K1 counted once per distinct (right block, input block))."""
    W = workers or (os.cpu_count() or 1)
    path, flops, total, desc = _oracle_sample(cfg_name, W)
    envv = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = _ORACLE_WORKER.replace("sys.path.insert(0, ROOT)", f"sys.path.insert(0, {ROOT!r})")
    procs = [subprocess.Popen([sys.executable, "-c", code, str(w), str(W), path, str(repeats), str(warmup)],
                              stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True, env=envv)
             for w in range(W)]
    try:
        for p in procs:
            line = p.stdout.readline()
            if not line.startswith("ready"):
                raise RuntimeError(p.stderr.read()[-2000:])
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        outs = []
        for p in procs:
            out, err = p.communicate(timeout=900)
            if p.returncode != 0:
                raise RuntimeError(err[-2000:])
            outs.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
        try:
            os.unlink(path)
        except OSError:
            pass
    per_rep = [max(d["times"][r] for d in outs) for r in range(repeats)]
    t = statistics.median(per_rep)
    return flops / t / 1e12, W, f"{desc}, median of {repeats}", t


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = synth.CONFIGS[args.config]
    v, cores, sample, t = oracle_cpu_baseline(args.config, max(1, args.steps), warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(cfg),
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--prec", default="split", choices=["fp64", "split"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slices", type=int, default=0,
                    help="BF16 slices per operand (0: picked by the library's autotuner)")
    ap.add_argument("--split-tol", type=float, default=3e-11, help="autotuner tolerance vs six slices")
    ap.add_argument("--t-budget-mb", type=int, default=0, help="device MB for one term chunk (0: default)")
    ap.add_argument("--ab-initio-config", default="qc32",
                    help="configuration of the ab initio block (environment built from the seeded integrals)")
    ap.add_argument("--no-ab-initio", action="store_true", help="skip the ab initio block")
    ap.add_argument("--out-of-core-config", default="qc64",
                    help="configuration of the out-of-core block (operators larger than the device)")
    ap.add_argument("--resident-gb", type=float, default=200.0,
                    help="GB of operator blocks kept on the device in the out-of-core block")
    ap.add_argument("--out-of-core-steps", type=int, default=2, help="timed H.psi of the out-of-core block")
    ap.add_argument("--no-out-of-core", action="store_true", help="skip the out-of-core block")
    ap.add_argument("--no-sweep", action="store_true", help="skip the sweep block")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2309_16724_gb300 as P
    from paper_2309_16724_gb300 import workload

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    cfg = synth.CONFIGS[args.config]
    prec = P.SU2_SPLIT_BF16 if args.prec == "split" else P.SU2_FP64
    ctx = P.Context(local, stream=stream)
    t0 = time.time()
    wall = {}  # seconds since the start of the bench at the end of each section

    def mark(name):
        wall[name] = round(time.time() - t0, 1)
    split = prec == P.SU2_SPLIT_BF16
    tune = split and args.slices == 0
    sec, env = workload.build(ctx, cfg, prepare_split=split, n_slices=args.slices,
                              t_budget_bytes=args.t_budget_mb << 20, autotune=tune, split_tol=args.split_tol)
    build_s = time.time() - t0
    n = sec.psi_len
    psi = torch.from_numpy(synth.gaussian_psi(n, synth.psi_seed(cfg))).to(dev)
    out = torch.empty_like(psi)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    info = env.info
    flops = info["flops_su2"]

    def status_ok(where):
        """The device status word after a section: a bounded device wait that
        gave up makes the bench fail instead of reporting a faster, aborted run."""
        st = ctx.status()
        if st:
            raise RuntimeError(f"device status {st} after {where}: a bounded device wait gave up")

    # the split result before any timing; the last timed step must reproduce
    # it bit for bit (the path is deterministic: no atomics in the sums)
    first = None
    if split:
        P.apply_heff(ctx, env, psi, out, prec)
        torch.cuda.synchronize()
        first = out.clone()
    for _ in range(args.warmup):
        P.apply_heff(ctx, env, psi, out, prec)
    torch.cuda.synchronize()
    status_ok("warm-up")
    env.profile(True)
    env.profile_reset()
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.apply_heff(ctx, env, psi, out, prec)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    status_ok("the timed steps")
    repeat_identical = bool(torch.equal(out, first)) if first is not None else None
    if first is not None and not repeat_identical:
        raise RuntimeError("the last timed H.psi differs from the first one")
    step_ms = [a.elapsed_time(b) for a, b in evs]
    tot_ms = sum(step_ms)
    prof = env.profile_read()
    env.profile(False)
    if world > 1:
        t = torch.tensor([tot_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = world * args.steps * flops / (tot_ms / 1e3) / 1e12

    # end to end through the C-ABI with host buffers (copies inside the call)
    e2e_steps = max(1, min(args.steps, 5))
    hin = torch.from_numpy(synth.gaussian_psi(n, synth.psi_seed(cfg))).pin_memory()
    hout = torch.empty(n, dtype=torch.float64).pin_memory()
    P.apply_heff_host(ctx, env, hin.numpy(), hout.numpy(), prec)
    e2e_t = []
    for _ in range(e2e_steps):
        t1 = time.perf_counter()
        P.apply_heff_host(ctx, env, hin.numpy(), hout.numpy(), prec)
        e2e_t.append(time.perf_counter() - t1)
    status_ok("the end-to-end steps")
    e2e_tot = sum(e2e_t)
    if world > 1:
        t = torch.tensor([e2e_tot], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t.item())
    e2e_value = world * e2e_steps * flops / e2e_tot / 1e12

    # one Davidson iteration (H.psi + FP64 Gram-Schmidt, Rayleigh-Ritz, residual,
    # correction), eager and as a CUDA-graph replay; host-timed (each step
    # returns theta and the residual norm to the host)
    dav_ms = {}
    for graph in (False, True):
        d = P.Davidson(ctx, env, psi, tol=1e-14, max_sub=24, keep=2, max_iter=1000, prec=prec, use_graph=graph)
        d.step()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(2):
            d.step()
        dav_ms["iter_ms_graph" if graph else "iter_ms_eager"] = (time.perf_counter() - t1) / 2 * 1e3
        d.close()
    status_ok("the Davidson steps")

    mark("main_environment_and_timed_sections")
    # the native-FP64 path on the same workload: a term shard (the operator
    # terms dealt to shards in longest-processing-time order of their flops),
    # timed with CUDA events; its rate is the shard's flops over its time.
    # On the same shard, the split H.psi against the FP64 one.
    # roofline inputs of the main environment before it may be released
    launch_count = prof.pop("kernel_launches")[0]
    fp64 = None
    rel_err_fp64 = None
    if split and rank == 0:
        n_sh = max(1, int(round(flops / 4e12)))
        if n_sh > 1:
            env.close()   # the shard's environment needs the memory (all timed sections are done)
            torch.cuda.synchronize()
            _, senv = workload.build(ctx, cfg, prepare_split=True, n_slices=info["split_slices"], shard=(0, n_sh))
        else:
            senv = env
        sfl = senv.info["flops_su2"]
        y64 = torch.empty_like(psi)
        ysp = torch.empty_like(psi)
        P.apply_heff(ctx, senv, psi, y64, P.SU2_FP64)
        P.apply_heff(ctx, senv, psi, ysp, P.SU2_SPLIT_BF16)
        torch.cuda.synchronize()
        rel_err_fp64 = float(torch.linalg.norm(ysp - y64) / torch.linalg.norm(y64))
        fms = []
        for _ in range(2):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            P.apply_heff(ctx, senv, psi, y64, P.SU2_FP64)
            b.record(stream)
            torch.cuda.synchronize()
            fms.append(a.elapsed_time(b))
        status_ok("the FP64-path steps")
        fv = sfl / (statistics.median(fms) / 1e3) / 1e12
        fp64 = {"value": fv, "unit": "TFLOP/s", "ms_per_step_sample": statistics.median(fms),
                "sample": (f"term shard 0 of {n_sh} ({100 * sfl / flops:.1f} % of the H.psi flops), "
                           "median of 2 timed H.psi after one untimed" if n_sh > 1 else
                           "the whole H.psi, median of 2 timed after one untimed"),
                "split_over_fp64": value / world / fv,
                "frac_of_nominal_fp64": fv / FP64_PEAK_TFLOPS}
        if senv is not env:
            senv.close()

    mark("fp64_path")
    # the ab initio Hamiltonian of the seeded integrals (Eq. 1): block
    # operators renormalised on the GPU (timed), split and FP64 H.psi, the
    # split error, and the split Davidson energy against the FP64 Rayleigh
    # quotient of the same vector
    ab = None
    if split and rank == 0 and not args.no_ab_initio:
        try:
            acfg = synth.CONFIGS[args.ab_initio_config]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            asec, aenv = workload.build(ctx, acfg, model=P.SU2_MODEL_AB_INITIO, prepare_split=True,
                                        n_slices=info["split_slices"])
            torch.cuda.synchronize()
            abuild = time.perf_counter() - t1
            ai = aenv.info
            apsi = torch.from_numpy(synth.gaussian_psi(asec.psi_len, synth.psi_seed(acfg))).to(dev)
            d = P.Davidson(ctx, aenv, apsi, tol=1e-8, max_iter=300, prec=P.SU2_SPLIT_BF16)
            th_s, res_s, it_s, conv = d.solve()
            x = torch.empty_like(apsi)
            d.vector(x)
            d.close()
            ys = torch.empty_like(apsi)
            y64 = torch.empty_like(apsi)
            times = {}
            for prec_, out_ in ((P.SU2_SPLIT_BF16, ys), (P.SU2_FP64, y64)):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                P.apply_heff(ctx, aenv, x, out_, prec_)
                b.record(stream)
                torch.cuda.synchronize()
                times[prec_] = a.elapsed_time(b)
            status_ok("the ab initio block")
            rq = float(torch.dot(x, y64) / torch.dot(x, x))
            res64 = float(torch.linalg.norm(y64 - rq * x) / torch.linalg.norm(x))
            afl = ai["flops_su2"]
            ab = {"workload": acfg.name, "L": acfg.L, "N": acfg.N, "D": acfg.D,
                  "operators": "ab initio from the seeded integrals, renormalised on the GPU",
                  "terms": ai["n_terms"], "tasks": ai["n_tasks"], "flops_su2_per_step": afl,
                  "env_build_s": abuild, "renorm_flops": ai["renorm_flops"],
                  "renorm_tflops": ai["renorm_flops"] / abuild / 1e12,
                  "split_tflops": afl / (times[P.SU2_SPLIT_BF16] / 1e3) / 1e12,
                  "fp64_tflops": afl / (times[P.SU2_FP64] / 1e3) / 1e12,
                  "split_over_fp64": times[P.SU2_FP64] / times[P.SU2_SPLIT_BF16],
                  "rel_err_split_vs_fp64": float(torch.linalg.norm(ys - y64) / torch.linalg.norm(y64)),
                  "davidson": {"energy_split": th_s, "iterations": it_s, "residual_split": res_s,
                               "converged": bool(conv), "rayleigh_quotient_fp64": rq,
                               "residual_fp64": res64, "dE_split_vs_fp64": th_s - rq,
                               "note": "split-precision Davidson to residual 1e-8; the FP64 Rayleigh quotient of "
                                       "its vector differs from the FP64 ground-state energy by O(residual^2)"}}
            aenv.close()
            asec.close()
        except Exception as ex:  # reported, not fatal
            ab = {"workload": args.ab_initio_config, "failed": str(ex)}

    mark("ab_initio")
    # out-of-core operators at the scale configuration: more operator bytes
    # than the device holds; the blocks beyond the resident budget lie in
    # pinned host memory and every H.psi streams them per term chunk
    ooc = None
    if split and rank == 0 and not args.no_out_of_core:
        try:
            ocfg = synth.CONFIGS[args.out_of_core_config]
            _, dev_total = torch.cuda.mem_get_info()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            osec, oenv_ = workload.build(ctx, ocfg, prepare_split=True, n_slices=info["split_slices"],
                                         resident_bytes=int(args.resident_gb * 1e9))
            torch.cuda.synchronize()
            obuild = time.perf_counter() - t1
            oi = oenv_.info
            opsi = torch.from_numpy(synth.gaussian_psi(osec.psi_len, synth.psi_seed(ocfg))).to(dev)
            oy = torch.empty_like(opsi)
            P.apply_heff(ctx, oenv_, opsi, oy, P.SU2_SPLIT_BF16)  # untimed
            ots = []
            for _ in range(max(1, args.out_of_core_steps)):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                P.apply_heff(ctx, oenv_, opsi, oy, P.SU2_SPLIT_BF16)
                b.record(stream)
                torch.cuda.synchronize()
                ots.append(a.elapsed_time(b))
            status_ok("the out-of-core block")
            oms = float(np.median(ots))
            ofl = oi["flops_su2"]
            ooc = {"workload": ocfg.name, "L": ocfg.L, "N": ocfg.N, "D": ocfg.D,
                   "operators": "synthetic-entry environments; the resident split path would need the FP64 "
                                "operators and their BF16 slices, about twice the device memory",
                   "operator_gb": oi["env_bytes"] / 1e9, "device_gb": dev_total / 1e9,
                   "resident_gb": oi["resident_bytes"] / 1e9, "streamed_gb_per_step": oi["streamed_bytes"] / 1e9,
                   "term_chunks": oi["n_io_chunks"], "tasks": oi["n_tasks"], "flops_su2_per_step": ofl,
                   "env_build_s": obuild, "steps": len(ots), "ms_per_step": oms,
                   "split_tflops": ofl / (oms / 1e3) / 1e12,
                   "io_gbs": oi["streamed_bytes"] / (oms / 1e3) / 1e9,
                   "note": "median of the timed split H.psi after one untimed; every H.psi copies the streamed "
                           "blocks host to device on the environment's IO stream, overlapped with compute"}
            oenv_.close()
            osec.close()
        except Exception as ex:  # reported, not fatal
            ooc = {"workload": args.out_of_core_config, "failed": str(ex)}

    mark("out_of_core")
    # two-site sweeps with wavefunction prediction on the split path: the
    # Heisenberg chain L = 12, D = 32, four sweeps (every window from the
    # second half-sweep on holds the ground state), and the L = N = 16 ab
    # initio Hamiltonian of the seeded integrals, D = 512, one full sweep
    sweeps = None
    if split and rank == 0 and not args.no_sweep:
        sweeps = {}
        for name, n_steps in (("heis12", 8 * 11), ("qc16", 2 * 15)):
            try:
                scfg = synth.CONFIGS[name]
                chain = synth.bond_sector_chain(scfg, scfg.L - 2)
                if scfg.site_kind == synth.SPIN_HALF:
                    hh = ee = None
                else:
                    hh, ee = synth.integrals(scfg.L, scfg.seed)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                sw = P.Sweep(ctx, hh, ee, chain, scfg.N, scfg.D, prec=P.SU2_SPLIT_BF16, tol=1e-8, seed=scfg.seed,
                             predict=True)
                e, w, it, _ = sw.run(n_steps, stats=True)
                sw.close()
                torch.cuda.synchronize()
                status_ok(f"the {name} sweep")
                half = scfg.L - 1
                sweeps[name] = {"L": scfg.L, "N": scfg.N, "D": scfg.D, "windows": n_steps,
                                "half_sweeps": n_steps // half, "s": time.perf_counter() - t1,
                                "davidson_iterations": int(it.sum()), "energy_last": float(e[-1]),
                                "energy_min": float(e.min()),
                                "energy_end_of_each_half_sweep": [float(x) for x in e[half - 1::half]],
                                "max_discarded_weight": float(w.max()),
                                "operators": ("Heisenberg, J = 1" if hh is None else
                                              "ab initio from the seeded integrals, renormalised on the GPU")}
            except Exception as ex:  # reported, not fatal
                sweeps[name] = {"failed": str(ex)}

    mark("sweeps")
    # roofline of the dominant kernel
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, ms, fl) = dom
    pk, src = peaks()
    if name.endswith("fp64"):
        bound, peak, unit = "alu", FP64_PEAK_TFLOPS, "TFLOP/s"
        peak_note = "nominal FP64 rate from SM count x DFMA/clk x max clock"
    else:
        bound, unit = "tensor", "TFLOP/s"
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        peak_note = f"{src} bf16 dense (sustained)"
    achieved = (fl / launches) / (ms / launches / 1e3) / 1e12 if launches else 0.0
    gpu_launches = int(launch_count)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            v, cores, sample, _ = oracle_cpu_baseline(cfg.name, 2)
            cpu = {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample}
        except Exception as ex:  # reported, not fatal
            cpu = {"value": None, "unit": "TFLOP/s", "cores": 0, "kind": "oracle", "sample": f"failed: {ex}"}

    mark("cpu_baseline")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == P.SU2_FP64 else "bf16",
            "data": "synthetic",
            "config": workload_config(cfg),
            "path": {"prec": "fp64" if prec == P.SU2_FP64 else
                     "bf16 slices on tcgen05, fp32 accumulate (exact per 192-K chunk), float-float/fp64 recombine",
                     "psi_len": n, "terms": info["n_terms"], "tasks": info["n_tasks"],
                     "slices": info["split_slices"] if split else None,
                     "stage_k16": info["split_stage_k"] if split else None,
                     "autotuned": tune},
            "value_u1_equiv": value * info["r_d"],
            "flops_su2_per_step": flops,
            "rel_err_vs_fp64": rel_err_fp64,
            "repeat_bit_identical": repeat_identical,
            "fp64_path": fp64,
            "ab_initio": ab,
            "out_of_core": ooc,
            "sweeps": sweeps,
            "wall_s": wall,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                    "steps": e2e_steps},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                         "frac": achieved / peak if peak else None,
                         "traffic": (k2_traffic(cfg.name, info["split_slices"], info["split_stage_k"])
                                     if name == "k2_split" else None),
                         "kernel": name, "peak_source": peak_note},
            "kernels": {k: {"launches": v[0], "ms": v[1], "flops": v[2]} for k, v in prof.items() if v[0]},
            "gpu_launches": gpu_launches,
            "davidson": dav_ms,
            "clocks": clk,
            "cpu_baseline": cpu,
            "build_s": build_s,
            "hbm_gb_in_use": round((torch.cuda.mem_get_info(dev)[1] - torch.cuda.mem_get_info(dev)[0]) / 1e9, 1),
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
