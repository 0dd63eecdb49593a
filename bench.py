"""Benchmark: eigenpairs/s of mixed-precision MRRR on one or more GB300s.

Workload (one step): the three n = 4001 tridiagonals of the mixed
single/double configuration -- 1-2-1 Toeplitz, Wilkinson W_4001 and Clement --
float32 in/out with binary64 internals, all eigenpairs, the three matrices in
one mrrr_solve_batch_s call (each solved on its own, Algorithm 1 per matrix,
in one sequence of launches).  Inputs are resident on the device; L2 is
flushed (256 MiB write) between timed steps.  Also reported: the same step as
three sequential and as three concurrent mrrr_solve_s calls, the 4096-matrix
batched workload, the double-double glued-Wilkinson solve and a bounded
replay of the serving trace.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank solves its own copy of the workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "eigenpairs/s (mixed-precision MRRR, all pairs)"
UNIT = "eigenpairs/s"
WORKLOAD = "3 x n=4001 tridiagonals (1-2-1, Wilkinson W_4001, Clement), fp32 in/out, fp64 internals, all eigenpairs"
# FP64 peak of one GB300: 152 SMs x 2 FP64 FMA units x 2 flop x 2070 MHz
# (matches the 1.25 TFLOP/s nominal figure; a DFMA loop measured 1194 GFLOP/s at 1987 MHz)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# algorithmic flops per counted qd step (one row of one transform)
FLOPS_PER_STEP = {"bisect": 4.0, "refine": 4.0, "rqi": 7.5, "shift": 5.0}
PHASE_COUNTER = {"bisect": "qd_bisect", "refine": "qd_refine", "rqi": "qd_rqi", "shift": "qd_shift"}
PHASE_KERNEL = {"bisect": "k_bisect", "refine": "k_bisect", "rqi": "k_rqi", "shift": "k_shift"}
# DRAM bytes (read + write) per k_rqi launch on this workload, the mean over the
# launches of one `ncu --set full` capture; valid only while the sources that
# define the kernel hash to the value they had at the capture
RQI_TRAFFIC = {"bytes_per_launch": 957.5e6, "sources_sha1": "f3d9c7e46fcc1075247d9a306e54fe13a65897d2",
               "sources": ("mrrr_core.cuh", "mrrr_dd.cuh", "mrrr_fast.cuh", "mrrr_phases.cuh", "mrrr_solver.cuh",
                           "mrrr_types.cuh", "solver_s.cu")}


def _rqi_traffic():
    import hashlib
    h = hashlib.sha1()
    for f in RQI_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_1304_1864_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return RQI_TRAFFIC["bytes_per_launch"] if h.hexdigest() == RQI_TRAFFIC["sources_sha1"] else None


def _workload():
    from paper_1304_1864_gb300 import inputs
    return [(np.asarray(d, np.float32), np.asarray(e, np.float32)) for d, e in inputs.workload_c2()]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # start timing only once the sampler reports (nvidia-smi takes a
            # moment to start), so that the samples cover the timed region
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _log(msg):
    sys.stderr.write("[bench %s] %s\n" % (time.strftime("%H:%M:%S"), msg))
    sys.stderr.flush()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ CPU oracle (reference arm and baseline)

def _oracle_sample(mats, per_matrix, threads=0):
    """Eigenpairs by the binary128 oracle for `per_matrix` evenly spaced
    indices of each matrix: Sturm bisection for the eigenvalue, inverse
    iteration for the vector.  Returns (pairs, seconds, threads)."""
    import oracle
    t0 = time.perf_counter()
    pairs = 0
    for d, e in mats:
        d64, e64 = d.astype(np.float64), e.astype(np.float64)
        n = d64.size
        for j in np.linspace(1, n, per_matrix).astype(int):
            hi, lo = oracle.eigvals(d64, e64, int(j), int(j), nthreads=threads)
            oracle.eigvecs(d64, e64, hi, lo)
            pairs += 1
    return pairs, time.perf_counter() - t0, oracle.max_threads() if threads == 0 else threads


def _oracle_bisect_sample(mats, per_matrix):
    """Eigenvalues only (all threads): per_matrix consecutive indices of each matrix."""
    import oracle
    t0 = time.perf_counter()
    cnt = 0
    for d, e in mats:
        d64, e64 = d.astype(np.float64), e.astype(np.float64)
        n = d64.size
        il = n // 2 - per_matrix // 2
        oracle.eigvals(d64, e64, il, il + per_matrix - 1)
        cnt += per_matrix
    return cnt, time.perf_counter() - t0


def cpu_baseline(mats, budget_s=12.0):
    """The oracle as it stands on this host: eigenvalue bisection in parallel
    over indices plus one inverse-iteration vector per index, on a sample
    sized for about `budget_s` seconds."""
    import oracle
    per = 8
    cnt, t = _oracle_bisect_sample(mats, per)
    while t < budget_s / 3 and per < 4096:
        per *= 2
        cnt, t = _oracle_bisect_sample(mats, per)
    # vectors for a small subset (inverse iteration, sequential)
    pv, tv, _ = _oracle_sample(mats, 2, threads=1)
    # eigenpair time = eigenvalue time (parallel) + vector time (per pair, sequential -> divide by threads)
    thr = oracle.max_threads()
    t_pair = t / cnt + max(tv / pv - t / cnt * thr, 0.0) / thr
    return {"value": 1.0 / t_pair, "unit": UNIT, "cores": thr, "kind": "oracle",
            "sample": "binary128 oracle: %d eigenvalues by Sturm bisection (%d threads, %.1f s) + %d "
                      "inverse-iteration vectors (%.1f s), middle of the spectrum of each n=4001 matrix; "
                      "eigenpairs/s = 1 / per-pair time" % (cnt, thr, t, pv, tv)}


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return 0
    mats = _workload()
    import oracle
    per = 2
    for _ in range(args.warmup):
        _oracle_sample(mats, per)
    tot_pairs, tot_t = 0, 0.0
    for _ in range(args.steps):
        p, t, thr = _oracle_sample(mats, per)
        tot_pairs += p
        tot_t += t
    value = tot_pairs / tot_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": "%d eigenpairs (bisection + inverse iteration) "
                       "per matrix, evenly spaced indices" % per},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "%d eigenpairs per step, single thread per pair" % (3 * per)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm

def _concurrent(fns):
    """Run the callables on their own host threads (the C ABI releases the
    interpreter lock) and re-raise the first failure."""
    errs = []

    def wrap(f):
        try:
            f()
        except BaseException as ex:  # noqa: BLE001 - reported below
            errs.append(ex)

    ts = [threading.Thread(target=wrap, args=(f,)) for f in fns]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if errs:
        raise errs[0]


class _Solo:
    """The C2 step: each matrix solved on its own by one mrrr_solve_s call,
    the three calls issued concurrently on three CUDA streams from three host
    threads, ordered after / before the caller's stream."""

    def __init__(self, m, mats, dev):
        import torch
        self.m, self.mats, self.dev = m, mats, dev
        self.streams = [torch.cuda.Stream(dev) for _ in mats]
        self.stats = [None] * len(mats)

    def run(self, timing=False):
        import torch
        main = torch.cuda.current_stream(self.dev)
        for s in self.streams:
            s.wait_stream(main)

        def one(i):
            d, e = self.mats[i]
            with torch.cuda.stream(self.streams[i]):
                W, Z, st = self.m.solve(d, e, mode="mixed", timing=timing, check=False)
            assert st["status"] == 0, st["status"]
            self.stats[i] = st

        _concurrent([lambda i=i: one(i) for i in range(len(self.mats))])
        for s in self.streams:
            main.wait_stream(s)
        return [dict(st) for st in self.stats]


class _Batch:
    """The C2 step: the three matrices in one mrrr_solve_batch_s call (each
    matrix solved on its own, Algorithm 1 per matrix, in one sequence of
    launches over all of them), on the caller's stream."""

    def __init__(self, m, mats):
        self.m, self.mats = m, mats

    def run(self, timing=False):
        out, st, status = self.m.solve_batch(self.mats, mode="mixed", timing=timing, check=False)
        assert all(s == 0 for s in status), status
        return [dict(st)]


def _time_steps(fn, steps, dev, flush):
    """Device time (ms) of `steps` calls of fn(), an L2 flush before each;
    returns (total ms, results)."""
    import torch
    stream = torch.cuda.current_stream(dev)
    total = 0.0
    out = []
    for _ in range(steps):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out.append(fn())
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    return total, out


PHASES_L = ("prep", "root", "bisect", "classify", "shift", "refine", "rqi", "finish")


def run_ours(args):
    import torch
    rank, world, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_1304_1864_gb300 as m
    m.lib()
    mats_h = _workload()
    mats = [(torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev)) for d, e in mats_h]
    pairs_per_step = sum(d.shape[0] for d, _ in mats_h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    step = _Batch(m, mats)
    for _ in range(args.warmup):
        step.run()
    torch.cuda.synchronize(dev)
    _barrier(world)
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        _barrier(world)
        ms_total, outs = _time_steps(lambda: step.run(timing=True), args.steps, dev, flush)
        torch.cuda.synchronize(dev)
        _barrier(world)
    acc = {}
    launches = 0
    for sts in outs:
        for st in sts:
            launches += sum(st["phase_launches"].values())
            for k in PHASES_L:
                acc["ms_" + k] = acc.get("ms_" + k, 0.0) + st["phase_ms"][k]
                acc["n_" + k] = acc.get("n_" + k, 0) + st["phase_launches"][k]
            for k in ("qd_bisect", "qd_refine", "qd_rqi", "qd_shift"):
                acc[k] = acc.get(k, 0) + st[k]
    last = outs[-1]
    ms_max = _max_over_ranks(ms_total, world, dev)
    value = pairs_per_step * args.steps * world / (ms_max / 1e3)
    # dominant kernel and its roofline (FP64 ALU bound); every launch is timed
    # with CUDA events on the stream it runs on
    phase_ms = {k: acc["ms_" + k] for k in PHASES_L}
    dom = max(PHASE_COUNTER, key=lambda p: phase_ms.get(p, 0.0))
    flops = acc[PHASE_COUNTER[dom]] * FLOPS_PER_STEP[dom]
    launches_dom = acc["n_" + dom]
    achieved = flops / (phase_ms[dom] / 1e3) / 1e9 if phase_ms[dom] > 0 else 0.0
    traffic = _rqi_traffic() if PHASE_KERNEL[dom] == "k_rqi" else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
                "traffic_note": ("bytes per launch, mean of the launches of one ncu capture of this kernel on this "
                                 "workload" if traffic else "kernel changed since the last ncu capture"),
                "kernel": PHASE_KERNEL[dom],
                "phase": dom, "launches": launches_dom,
                "ms_per_launch": phase_ms[dom] / max(launches_dom, 1),
                "flops_per_launch": flops / max(launches_dom, 1),
                "peak_note": "of derived FP64 peak: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz (the measured "
                             "peaks file has no FP64 figure; a DFMA loop measured 1194 GFLOP/s)",
                "phase_share": {k: v / max(sum(phase_ms.values()), 1e-30) for k, v in phase_ms.items()}}
    line = None
    if rank == 0:
        _log("timed steps: %.1f ms" % ms_total)
        e2e = _e2e(m, mats_h, args, dev)
        _log("e2e done")
        cb = cpu_baseline(mats_h) if (world == 1 and not args.no_cpu_baseline) else None
        _log("cpu baseline done")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "mode": "mixed single/double (fp32 io, fp64 internals)",
                           "solves": "the 3 matrices in one mrrr_solve_batch_s call: each matrix solved on its "
                                     "own (Algorithm 1 per matrix) in one sequence of launches over all of them",
                           "l2": "flushed (256 MiB write) between timed steps", "parallelism": "replica per GPU"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(),
                "tree": {nm: last[0][key] for nm, key in
                         (("d_max", "d_max"), ("clusters", "nclusters"), ("largest_cluster", "largest_cluster"),
                          ("reps_failed", "reps_failed"), ("rqi_iters", "rqi_iters"), ("fallbacks", "fallbacks"))}}
        line["variants"] = _variants(m, mats, args, dev, flush)
        if not args.no_extras:
            for key, fn in (("c4_batched", lambda: _c4(m, dev, flush)),
                            ("c3_dd", lambda: _c3(m, dev, flush)),
                            ("serve", lambda: _serve(m, dev, args.serve_requests))):
                t0 = time.perf_counter()
                line[key] = fn()
                _log("%s: %.1f s" % (key, time.perf_counter() - t0))
        if args.plain:
            line["plain"] = _plain(m, mats, args, dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _variants(m, mats, args, dev, flush):
    """The same C2 step issued as three sequential mrrr_solve_s calls and as
    three concurrent ones (three streams, three host threads)."""
    import torch
    pairs = sum(d.shape[0] for d, _ in mats)
    res = {}

    def seq():
        for d, e in mats:
            m.solve(d, e, mode="mixed", check=True)

    solo = _Solo(m, mats, dev)

    for label, fn in (("sequential_solves", seq), ("concurrent_solves", solo.run)):
        fn()
        torch.cuda.synchronize(dev)
        ms, _ = _time_steps(fn, args.steps, dev, flush)
        res[label] = {"value": pairs * args.steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / args.steps}
    return res


def _c4(m, dev, flush):
    """Batched workload: 4096 tridiagonals, n log-uniform in [32, 2048], types
    {U(-1,1), 1-2-1, Wilkinson, glued W_21 (coupling 1e-8)}, fp32 in, fp64
    internals, all eigenpairs, one mrrr_solve_batch_s call; one warm-up call
    and one timed call."""
    import torch
    from paper_1304_1864_gb300 import inputs
    batch = inputs.workload_c4(count=4096, seed=4)
    mats = [(torch.tensor(d, dtype=torch.float32, device=dev), torch.tensor(e, dtype=torch.float32, device=dev))
            for _, d, e in batch]
    pairs = sum(d.size for _, d, _ in batch)

    def step():
        out, st, status = m.solve_batch(mats, mode="mixed")
        assert all(s == 0 for s in status)
        return st

    step()
    torch.cuda.synchronize(dev)
    ms, sts = _time_steps(step, 1, dev, flush)
    st = sts[0]
    return {"value": pairs / (ms / 1e3), "unit": UNIT, "ms": ms, "matrices": len(batch), "eigenpairs": pairs,
            "d_max": st["d_max"], "clusters": st["nclusters"], "fallbacks": st["fallbacks"],
            "workload": "4096 tridiagonals, n log-uniform [32, 2048], seed 4, types uniform/1-2-1/Wilkinson/"
                        "glued W_21, fp32 in, fp64 internals, all pairs, one batched call"}


def _c3(m, dev, flush):
    """Glued Wilkinson, 40 x W_201 with couplings 1e-8 (n = 8040), fp64 in,
    double-double internals, all eigenpairs; one warm-up and one timed solve."""
    import torch
    from paper_1304_1864_gb300 import inputs
    (d, e), = inputs.workload_c3()
    dd = torch.tensor(d, dtype=torch.float64, device=dev)
    ee = torch.tensor(e, dtype=torch.float64, device=dev)
    m.solve(dd, ee, mode="mixed")
    torch.cuda.synchronize(dev)
    ms, sts = _time_steps(lambda: m.solve(dd, ee, mode="mixed")[2], 1, dev, flush)
    st = sts[0]
    return {"value": d.size / (ms / 1e3), "unit": UNIT, "ms": ms, "n": int(d.size), "d_max": st["d_max"],
            "clusters": st["nclusters"], "largest_cluster": st["largest_cluster"],
            "workload": "glued Wilkinson 40 x W_201, couplings 1e-8, n=8040, fp64 in, double-double internals"}


def _serve(m, dev, count):
    """Serving loop: the first `count` requests of the seeded Poisson trace
    (2000 requests/s, n log-uniform [64, 16384], half fp32 in with fp64
    internals, half fp64 in with double-double internals, half all pairs, half
    a random contiguous 10% index range), submitted at their arrival times
    (host inputs, device outputs) to one server; latency is submit to
    completion."""
    import torch
    from paper_1304_1864_gb300 import inputs
    trace = inputs.serving_trace(rate=2000.0, seconds=1.0, seed=5)[:count]
    reqs = []
    for r in trace:
        d, e = inputs.make(r["kind"], r["n"], seed=int(r["t"] * 1e6) % (2**31))
        n = d.size
        if r["il"] == 1 and r["iu"] == r["n"]:
            il, iu = 0, 0
        else:
            il = min(r["il"], n)
            iu = max(il, min(r["iu"], n))
        npdt = np.float32 if r["prec"] == "s" else np.float64
        reqs.append((r["t"], d.astype(npdt), (e if n > 1 else np.zeros(1)).astype(npdt), il, iu, r["prec"]))
    srv = m.Server(workers=3)
    try:
        keep = {}
        t0 = time.perf_counter()
        for t, d, e, il, iu, prec in reqs:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            n = d.size
            k = (iu - il + 1) if il else n
            tdt = torch.float32 if prec == "s" else torch.float64
            W = torch.empty(k, dtype=tdt, device=dev)
            Z = torch.empty((k, n), dtype=tdt, device=dev)
            tk = srv.submit(d, e, W, Z, mode="mixed", il=il, iu=iu)
            keep[tk] = (W, Z)
        bad = 0
        for tk in list(keep):
            rc, info = srv.poll(tk, wait_ms=-1)
            bad += rc != 0
            del keep[tk]
        wall = time.perf_counter() - t0
        st = srv.stats()
    finally:
        srv.close()
    return {"requests": len(reqs), "failed": bad, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "max_ms": st["max_ms"], "eigenpairs": st["eigenpairs"], "batches": st["batches"],
            "value": st["eigenpairs"] / max(st["busy_s"], 1e-9), "unit": UNIT, "wall_s": wall,
            "offered": "Poisson 2000 requests/s (trace seed 5), first %d requests replayed at their arrival times; "
                       "n log-uniform [64, 16384]; half fp32->fp64, half fp64->double-double; half all pairs, "
                       "half 10%% index ranges; 3 workers, budget = half the free HBM" % len(reqs)}


def _plain(m, mats, args, dev):
    """Plain MRRR (working precision = I/O precision: fp32) and the plain
    FP64 solver run on the same fp32 data as fp64 input, for comparison."""
    import torch
    res = {}
    for label, mm, mode in (("plain_fp32", mats, "plain"),
                            ("plain_fp64", [(d.double(), e.double()) for d, e in mats], "plain")):
        for _ in range(2):
            m.solve_batch(mm, mode=mode)
        torch.cuda.synchronize(dev)
        t = 0.0
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            m.solve_batch(mm, mode=mode)
            b.record()
            b.synchronize()
            t += a.elapsed_time(b)
        res[label] = {"value": sum(d.shape[0] for d, _ in mm) * args.steps / (t / 1e3), "unit": UNIT}
    return res


def _e2e(m, mats_h, args, dev):
    """The C2 step end to end through the public API, as the headline step
    (one mrrr_solve_batch_s call through the binding's solve_batch): each
    step copies the inputs from pinned host memory to the device, solves,
    and copies W and Z back to pinned host memory, all inside the timed
    region (wall clock, the stream synchronised at the end of every step)."""
    import torch
    pin_in = [(torch.from_numpy(d).pin_memory(), torch.from_numpy(e).pin_memory()) for d, e in mats_h]
    dev_in = [(torch.empty(d.shape, dtype=d.dtype, device=dev), torch.empty(e.shape, dtype=e.dtype, device=dev))
              for d, e in pin_in]
    pin_out = []
    stream = torch.cuda.current_stream(dev)

    def step():
        for (dh, eh), (dd, ed) in zip(pin_in, dev_in):
            dd.copy_(dh, non_blocking=True)
            ed.copy_(eh, non_blocking=True)
        out, st, status = m.solve_batch(dev_in, mode="mixed", check=False)
        assert all(s == 0 for s in status), status
        if not pin_out:
            for W, Z in out:
                pin_out.append((torch.empty(W.shape, dtype=W.dtype).pin_memory(),
                                torch.empty(Z.T.shape, dtype=Z.dtype).pin_memory()))
        for (W, Z), (Wh, Zh) in zip(out, pin_out):
            Wh.copy_(W, non_blocking=True)
            Zh.copy_(Z.T, non_blocking=True)
        stream.synchronize()

    for _ in range(max(1, args.warmup)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    pairs = sum(d.size for d, _ in mats_h)
    h2d = sum(4 * (d.size + e.size) for d, e in mats_h)
    d2h = sum(4 * (d.size + d.size * d.size) for d, _ in mats_h)
    return {"value": pairs * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "mrrr_solve_batch_s through the binding's solve_batch; inputs copied from pinned host memory and "
                   "W, Z copied back to pinned host memory inside the timed region"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain", action="store_true", help="also time the plain (y = x) solvers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, C3, C4 and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests replayed from the serving trace")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
