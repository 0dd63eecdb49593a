"""Benchmark: eigenpairs/s of mixed-precision MRRR on one or more GB300s.

Workload (one step): the three n = 4001 tridiagonals of the mixed
single/double configuration -- 1-2-1 Toeplitz, Wilkinson W_4001 and Clement --
float32 in/out with binary64 internals, all eigenpairs, each matrix an
independent problem, solved in one batched call.  Inputs are resident on the
device; L2 is flushed (256 MiB write) between timed steps.

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
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        m.solve_batch(mats, mode="mixed")
    torch.cuda.synchronize(dev)
    _barrier(world)
    stats_acc = {}
    launches = 0
    ms_total = 0.0
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize(dev)
        _barrier(world)
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            out, st, status = m.solve_batch(mats, mode="mixed", timing=True)
            b.record(stream)
            b.synchronize()
            assert all(s == 0 for s in status), status
            ms_total += a.elapsed_time(b)
            launches += sum(st["phase_launches"].values())
            for k, v in st["phase_ms"].items():
                stats_acc.setdefault("ms_" + k, 0.0)
                stats_acc["ms_" + k] += v
            for k in ("qd_bisect", "qd_refine", "qd_rqi", "qd_shift"):
                stats_acc[k] = stats_acc.get(k, 0) + st[k]
            last_stats = st
        torch.cuda.synchronize(dev)
        _barrier(world)
    ms_max = _max_over_ranks(ms_total, world, dev)
    value = pairs_per_step * args.steps * world / (ms_max / 1e3)
    # dominant kernel and its roofline (FP64 ALU bound)
    phase_ms = {k[3:]: v for k, v in stats_acc.items() if k.startswith("ms_")}
    dom = max(PHASE_COUNTER, key=lambda p: phase_ms.get(p, 0.0))
    flops = stats_acc[PHASE_COUNTER[dom]] * FLOPS_PER_STEP[dom]
    launches_dom = last_stats["phase_launches"][dom] * args.steps
    achieved = flops / (phase_ms[dom] / 1e3) / 1e9 if phase_ms[dom] > 0 else 0.0
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None, "kernel": PHASE_KERNEL[dom],
                "phase": dom, "launches": launches_dom,
                "ms_per_launch": phase_ms[dom] / max(launches_dom, 1),
                "flops_per_launch": flops / max(launches_dom, 1),
                "peak_note": "FP64 FMA peak derived: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
                "phase_share": {k: v / max(sum(phase_ms.values()), 1e-30) for k, v in phase_ms.items()}}
    # end to end: the public C ABI with pinned host buffers, copies inside the timed region
    e2e = None
    if rank == 0:
        e2e = _e2e(m, mats_h, args, dev)
    line = None
    if rank == 0:
        cb = cpu_baseline(mats_h) if (world == 1 and not args.no_cpu_baseline) else None
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "mode": "mixed single/double (fp32 io, fp64 internals)",
                           "l2": "flushed (256 MiB write) between timed steps", "parallelism": "replica per GPU"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk.summary(), "tree": {"d_max": last_stats["d_max"], "clusters": last_stats["nclusters"],
                                                  "largest_cluster": last_stats["largest_cluster"],
                                                  "reps_failed": last_stats["reps_failed"],
                                                  "rqi_iters": last_stats["rqi_iters"],
                                                  "fallbacks": last_stats["fallbacks"]}}
        if args.plain:
            line["plain"] = _plain(m, mats, args, dev)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


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
    import ctypes
    import torch
    pin = []
    for d, e in mats_h:
        n = d.size
        dp = torch.from_numpy(d).pin_memory()
        ep = torch.from_numpy(e).pin_memory()
        W = torch.empty(n, dtype=torch.float32).pin_memory()
        Z = torch.empty((n, n), dtype=torch.float32).pin_memory()
        pin.append((n, dp, ep, W, Z))
    stream = torch.cuda.current_stream(dev)
    sh = ctypes.c_void_p(stream.cuda_stream)

    def step():
        for n, dp, ep, W, Z in pin:
            mcount = ctypes.c_int(0)
            rc = m.mrrr_solve_s(n, ctypes.c_void_p(dp.data_ptr()), ctypes.c_void_p(ep.data_ptr()), 0,
                                ctypes.c_float(0), ctypes.c_float(0), 1, n, 1, None, ctypes.byref(mcount),
                                ctypes.c_void_p(W.data_ptr()), ctypes.c_void_p(Z.data_ptr()), n, sh)
            assert rc == 0, rc

    for _ in range(max(1, args.warmup)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    pairs = sum(p[0] for p in pin)
    h2d = sum(4 * (2 * p[0] - 1) for p in pin)
    d2h = sum(4 * (p[0] + p[0] * p[0]) for p in pin)
    return {"value": pairs * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "mrrr_solve_s x3 with pinned host buffers (sequential calls)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain", action="store_true", help="also time the plain (y = x) solvers")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
