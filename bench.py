"""Benchmark: eigenpairs/s of mixed-precision MRRR on one or more GB300s.

Workload (one step): the three n = 4001 tridiagonals of the mixed
single/double configuration -- 1-2-1 Toeplitz, Wilkinson W_4001 and Clement --
float32 in/out with binary64 internals, all eigenpairs, the three matrices in
one mrrr_solve_batch_s call (each solved on its own, Algorithm 1 per matrix,
in one sequence of launches).  Inputs are resident on the device; L2 is
flushed (256 MiB write) between timed steps.  Also reported: plain MRRR
(binary32 and binary64 inside) on the same matrices with the residual and
orthogonality of every leg, the step end to end through the C ABI with host
buffers, the same step as three sequential and as three concurrent
mrrr_solve_s calls, the 4096-matrix batched workload, the double-double
glued-Wilkinson solve and a sweep of offered rates through the serving loop.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
--gpus N > 1 outside a distributed launcher starts N ranks through
torch.distributed.run.  Every rank solves its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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
# FP64 peak of one GB300 derived from unit counts and the clock: 152 SMs x 2
# FP64 FMA per clock per SM x 2 flop x 2070 MHz (the nominal 1.25 TFLOP/s)
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# Algorithmic flops of the Rayleigh quotient iteration (Algorithm 1, line 10;
# Sec. 2, "Rayleigh quotient iteration"), counted per row of the step's block:
# one step is the stationary and the progressive transform (3 flops each, the
# divides not counted) and gamma_k (2 flops) = 8 per row; forming the vector
# (recurrence, norm, scale) = 3 per row per eigenpair.  In double-double the
# same operations are counted as binary64 instructions with the multipliers
# add ~10, mul ~4, div ~17 (FMA-based TwoSum/TwoProd and long division): a
# step row has 6 adds, 2 muls and 2 divides = 102, a vector row 3 muls and 1
# add = 22.
RQI_FLOPS = {"f64": (8.0, 3.0), "dd": (102.0, 22.0)}
# DRAM bytes (read + write) per k_rqi launch on this workload, the mean over the
# launches of one `ncu --set full` capture; valid only while the sources that
# define the kernel hash to the value they had at the capture
RQI_TRAFFIC = {"bytes_per_launch": 935.12e6, "sources_sha1": "075ac0479d93b851d6f19eeec3cfdb9de873563b",
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
    """One step: the matrices in one mrrr_solve_batch call (each matrix solved
    on its own, Algorithm 1 per matrix, in one sequence of launches over all
    of them), on the caller's stream."""

    def __init__(self, m, mats, mode="mixed"):
        self.m, self.mats, self.mode = m, mats, mode
        self.last = None

    def run(self, timing=False):
        out, st, status = self.m.solve_batch(self.mats, mode=self.mode, timing=timing, check=False)
        assert all(s == 0 for s in status), status
        self.last = out
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


def _sum_stats(outs):
    """Phase times, launches and counters summed over the solves of the timed steps."""
    acc = {"launches": 0, "rqi_rows": 0, "rqi_iters": 0}
    for sts in outs:
        for st in sts:
            acc["launches"] += sum(st["phase_launches"].values())
            for k in PHASES_L:
                acc["ms_" + k] = acc.get("ms_" + k, 0.0) + st["phase_ms"][k]
                acc["n_" + k] = acc.get("n_" + k, 0) + st["phase_launches"][k]
            for k in ("qd_bisect", "qd_refine", "qd_rqi", "qd_shift", "rqi_rows", "rqi_iters"):
                acc[k] = acc.get(k, 0) + st[k]
    return acc


def _rqi_roofline(acc, pairs_rows, arith, peak_measured, traffic=None):
    """Roofline of k_rqi over the timed steps: algorithmic flops (RQI_FLOPS:
    per row of each RQI step, plus per row of each eigenpair's vector) over the
    summed CUDA-event time of its launches (on the streams they run on),
    against the derived FP64 peak (ALU bound; dd counted in binary64
    instructions) and against the measured DFMA rate."""
    per_step, per_vec = RQI_FLOPS[arith]
    flops = acc["rqi_rows"] * per_step + pairs_rows * per_vec
    ms = acc["ms_rqi"]
    launches = max(acc["n_rqi"], 1)
    achieved = flops / (ms / 1e3) / 1e9 if ms > 0 else 0.0
    phase_ms = {k: acc["ms_" + k] for k in PHASES_L}
    tot = max(sum(phase_ms.values()), 1e-30)
    return {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic,
            "kernel": "k_rqi<float, double>" if arith == "f64" else "k_rqi<double, dd>",
            "launches": acc["n_rqi"], "ms_per_launch": ms / launches, "flops_per_launch": flops / launches,
            "flop_count": "%g per row per RQI step (rqi_rows = %d) + %g per row per eigenpair (%d rows)" % (
                per_step, acc["rqi_rows"], per_vec, pairs_rows),
            "peak_note": "derived FP64 peak: 152 SMs x 2 DFMA/clk x 2 flop x 2070 MHz",
            "peak_measured_gflops": peak_measured,
            "frac_of_measured": achieved / peak_measured if peak_measured else None,
            "phase_share": {k: v / tot for k, v in phase_ms.items()}}


def _accuracy(pairs):
    """Largest residual ||T z - w z||_2 / (||T||_1 n eps_x) and orthogonality
    max |Z^T Z - I| / (n eps_x) over the solved matrices, evaluated on the
    device in binary64 (products of binary32 data are exact there; for
    binary64 data the accumulation error, about sqrt(n) eps_d, is far below
    the n eps_d unit).  pairs: list of (d, e, W, Z) device tensors."""
    import torch
    res, orth = 0.0, 0.0
    for d, e, W, Z in pairs:
        eps = 2.0 ** -24 if d.dtype == torch.float32 else 2.0 ** -53
        n = d.shape[0]
        d64, e64 = d.double(), e.double()
        Z64, W64 = Z.double(), W.double()
        TZ = d64[:, None] * Z64
        TZ[:-1] += e64[:, None] * Z64[1:]
        TZ[1:] += e64[:, None] * Z64[:-1]
        R = TZ - Z64 * W64[None, :]
        absd = d64.abs()
        rows = absd.clone()
        rows[:-1] += e64.abs()
        rows[1:] += e64.abs()
        tn = float(rows.max())
        res = max(res, float(R.norm(dim=0).max()) / (tn * n * eps))
        G = Z64.T @ Z64
        G.diagonal().sub_(1.0)
        orth = max(orth, float(G.abs().max()) / (n * eps))
    return res, orth


def _probe_peak(m):
    try:
        g, t = m.probe_fp64()
        return g, t
    except Exception as ex:  # noqa: BLE001 - reported in the line
        _log("fp64 probe failed: %s" % ex)
        return None, None


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
    peak_meas, peak_ms = (None, None) if args.step_only else _probe_peak(m)
    mats_h = _workload()
    mats = [(torch.from_numpy(d).to(dev), torch.from_numpy(e).to(dev)) for d, e in mats_h]
    pairs_per_step = sum(d.shape[0] for d, _ in mats_h)
    pair_rows = sum(d.shape[0] * d.shape[0] for d, _ in mats_h)
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
    acc = _sum_stats(outs)
    last = outs[-1]
    ms_max = _max_over_ranks(ms_total, world, dev)
    value = pairs_per_step * args.steps * world / (ms_max / 1e3)
    roofline = _rqi_roofline(acc, pair_rows * args.steps, "f64", peak_meas, _rqi_traffic())
    roofline["traffic_note"] = ("bytes per launch, mean of the launches of one ncu capture of this kernel on this "
                                "workload" if roofline["traffic"] else "kernel changed since the last ncu capture")
    line = None
    if rank == 0 and args.step_only:
        # only the timed steps (for launch lists and counter captures)
        print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "step_only": True,
                          "roofline": roofline, "gpu_launches": acc["launches"]}), flush=True)
    elif rank == 0:
        _log("timed steps: %.1f ms" % ms_total)
        comparison = _compare(m, mats, step, args, dev, flush, value)
        _log("plain comparison done")
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
                           "l2": "flushed (256 MiB write) between timed steps",
                           "parallelism": "replica per GPU" if world > 1 else "1 GPU"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "gpu_launches": acc["launches"],
                "clocks": clk.summary(),
                "fp64_probe": {"gflops": peak_meas, "ms": peak_ms,
                               "what": "mrrr_probe_fp64_fma: 8 warps per SM, 8 independent DFMA chains per thread"},
                "comparison": comparison,
                "tree": _tree(last[0])}
        line["variants"] = _variants(m, mats, args, dev, flush)
        if not args.no_extras:
            for key, fn in (("c4_batched", lambda: _c4(m, dev, flush, args, peak_meas)),
                            ("c3_dd", lambda: _c3(m, dev, flush, args, peak_meas)),
                            ("dense", lambda: _dense(m, dev, flush, args)),
                            ("serve", lambda: _serve(m, dev, args))):
                t0 = time.perf_counter()
                line[key] = fn()
                _log("%s: %.1f s" % (key, time.perf_counter() - t0))
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _tree(st):
    """Representation-tree statistics of one solve (Sec. 2 and 3.2)."""
    keys = ("d_max", "nclusters", "largest_cluster", "reps_failed", "reps_relaxed", "reps_backtracked",
            "rqi_iters", "fallbacks", "noconv")
    return {k: st[k] for k in keys}


def _compare(m, mats, step, args, dev, flush, value):
    """The metric's comparison: mixed precision against plain MRRR on the same
    three matrices -- plain binary32 (y = x, the same fp32 input) and the plain
    FP64-internal solver (y = x = binary64, the matrices given as fp64) --
    each as one batched call, timed like the headline step; then residual and
    orthogonality of each result in units of n eps of its own I/O precision."""
    import torch
    k = max(3, min(args.steps, 20))
    pairs = sum(d.shape[0] for d, _ in mats)
    res = {}
    legs = (("mixed_fp32_fp64", step, mats),
            ("plain_fp32", _Batch(m, mats, "plain"), mats),
            ("plain_fp64", _Batch(m, [(d.double(), e.double()) for d, e in mats], "plain"),
             [(d.double(), e.double()) for d, e in mats]))
    for label, st, mm in legs:
        if label != "mixed_fp32_fp64":
            for _ in range(2):
                st.run()
            torch.cuda.synchronize(dev)
            ms, _ = _time_steps(st.run, k, dev, flush)
            v = pairs * k / (ms / 1e3)
        else:
            v = value
            st.run()
        torch.cuda.synchronize(dev)
        r, o = _accuracy([(d, e, W, Z) for (d, e), (W, Z) in zip(mm, st.last)])
        res[label] = {"value": v, "unit": UNIT, "residual_neps": r, "orthogonality_neps": o}
    res["note"] = ("residual ||Tz - wz||_2 / (||T||_1 n eps_x) and orthogonality max|Z^T Z - I| / (n eps_x), "
                   "worst over the three matrices, eps_x of each leg's I/O precision; binary64 evaluation on the "
                   "device")
    return res


def _variants(m, mats, args, dev, flush):
    """The same C2 step issued as three sequential mrrr_solve_s calls and as
    three concurrent ones (three streams, three host threads)."""
    import torch
    pairs = sum(d.shape[0] for d, _ in mats)
    res = {}
    k = max(3, min(args.steps, 20))

    def seq():
        for d, e in mats:
            m.solve(d, e, mode="mixed", check=True)

    solo = _Solo(m, mats, dev)

    for label, fn in (("sequential_solves", seq), ("concurrent_solves", solo.run)):
        fn()
        torch.cuda.synchronize(dev)
        ms, _ = _time_steps(fn, k, dev, flush)
        res[label] = {"value": pairs * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k}
    return res


def _c4(m, dev, flush, args, peak_meas):
    """Batched workload: 4096 tridiagonals, n log-uniform in [32, 2048], types
    {U(-1,1), 1-2-1, Wilkinson, glued W_21 (coupling 1e-8)}, fp32 in, fp64
    internals, all eigenpairs, one mrrr_solve_batch_s call per step."""
    import torch
    from paper_1304_1864_gb300 import inputs
    batch = inputs.workload_c4(count=4096, seed=4)
    mats = [(torch.tensor(d, dtype=torch.float32, device=dev), torch.tensor(e, dtype=torch.float32, device=dev))
            for _, d, e in batch]
    pairs = sum(d.size for _, d, _ in batch)
    pair_rows = sum(d.size * d.size for _, d, _ in batch)
    step = _Batch(m, mats)
    step.run()
    torch.cuda.synchronize(dev)
    k = args.extra_steps
    ms, sts = _time_steps(lambda: step.run(timing=True), k, dev, flush)
    acc = _sum_stats(sts)
    st = sts[-1][0]
    return {"value": pairs * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
            "matrices": len(batch), "eigenpairs": pairs, "tree": _tree(st),
            "roofline": _rqi_roofline(acc, pair_rows * k, "f64", peak_meas),
            "workload": "4096 tridiagonals, n log-uniform [32, 2048], seed 4, types uniform/1-2-1/Wilkinson/"
                        "glued W_21, fp32 in, fp64 internals, all pairs, one batched call per step"}


def _c3(m, dev, flush, args, peak_meas):
    """Glued Wilkinson, 40 x W_201 with couplings 1e-8 (n = 8040), fp64 in,
    double-double internals, all eigenpairs, one mrrr_solve_d per step."""
    import torch
    from paper_1304_1864_gb300 import inputs
    (d, e), = inputs.workload_c3()
    dd = torch.tensor(d, dtype=torch.float64, device=dev)
    ee = torch.tensor(e, dtype=torch.float64, device=dev)
    m.solve(dd, ee, mode="mixed")
    torch.cuda.synchronize(dev)
    k = args.extra_steps
    ms, sts = _time_steps(lambda: [m.solve(dd, ee, mode="mixed", timing=True)[2]], k, dev, flush)
    acc = _sum_stats(sts)
    st = sts[-1][0]
    n = int(d.size)
    return {"value": n * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k, "n": n,
            "tree": _tree(st), "roofline": _rqi_roofline(acc, n * n * k, "dd", peak_meas),
            "workload": "glued Wilkinson 40 x W_201, couplings 1e-8, n=8040, fp64 in, double-double internals"}


def _dense(m, dev, flush, args):
    """The dense experiment of Sec. 5 (Fig. 3): A = Q T Q^T with T the n = 2000
    1-2-1 matrix and Q the orthogonal factor of a seeded Gaussian matrix,
    fp32 in/out; reduction to tridiagonal form, tridiagonal MRRR (mixed, and
    plain for comparison), back-transformation, all eigenpairs, one
    mrrr_syev_s call per step.  Residual ||A z - w z||_2 / (||A||_1 n eps) and
    orthogonality in units of n eps, evaluated on the device in binary64."""
    import torch
    from paper_1304_1864_gb300 import inputs
    n = 2000
    d, e = inputs.one_two_one(n)
    rng = np.random.default_rng(7)
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    Q *= np.sign(np.diag(R))
    A = Q @ (np.diag(d) + np.diag(e, 1) + np.diag(e, -1)) @ Q.T
    Ag = torch.tensor(0.5 * (A + A.T), dtype=torch.float32, device=dev)
    out = {"n": n, "workload": "A = Q T Q^T, T = 1-2-1 (n = 2000), Q from a seeded Gaussian matrix, fp32 in/out, "
                               "all eigenpairs, one mrrr_syev_s call per step"}
    for mode in ("mixed", "plain"):
        m.solve_dense(Ag, mode=mode)
        torch.cuda.synchronize(dev)
        k = max(1, min(args.extra_steps, 3))
        ms, sts = _time_steps(lambda: [m.solve_dense(Ag, mode=mode)], k, dev, flush)
        W, Z, st = sts[-1][0]
        A64, Z64, W64 = Ag.double(), Z.double(), W.double()
        R = A64 @ Z64 - Z64 * W64[None, :]
        an = float(A64.abs().sum(dim=0).max())
        eps = 2.0 ** -24
        G = Z64.T @ Z64
        G.diagonal().sub_(1.0)
        out[mode] = {"value": n * k / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
                     "residual_neps": float(R.norm(dim=0).max()) / (an * n * eps),
                     "orthogonality_neps": float(G.abs().max()) / (n * eps)}
    return out


def _serve_run(m, dev, trace):
    """Submit the requests of `trace` at their arrival times (host inputs,
    device outputs) to one server and wait for all; latency is submit to
    completion."""
    import torch
    from paper_1304_1864_gb300 import inputs
    reqs = []
    for r in trace:
        d, e = inputs.make(r["kind"], r["n"], seed=r["seed"])
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
            "value": st["eigenpairs"] / max(st["busy_s"], 1e-9), "unit": UNIT, "wall_s": wall}


def _serve(m, dev, args):
    """Serving loop (continuous batching) on the request mix of the serving
    trace -- n log-uniform [64, 16384], half fp32 in with fp64 internals and
    half fp64 in with double-double internals, half all pairs and half a
    random contiguous 10% index range -- at a sweep of Poisson arrival rates
    up to and past the server's capacity, each for a bounded window; then
    the first requests of the 2000 requests/s trace as the overload point."""
    from paper_1304_1864_gb300 import inputs
    sweep = []
    for rate in args.serve_rates:
        trace = inputs.serving_trace(rate=rate, seconds=args.serve_seconds, seed=5)
        r = _serve_run(m, dev, trace)
        r["offered_req_per_s"] = rate
        r["window_s"] = args.serve_seconds
        sweep.append(r)
        _log("serve %.1f req/s: %d requests, p50 %.0f ms, p99 %.0f ms" % (rate, r["requests"], r["p50_ms"],
                                                                            r["p99_ms"]))
    over = _serve_run(m, dev, inputs.serving_trace(rate=2000.0, seconds=1.0, seed=5)[:args.serve_requests])
    over["offered"] = ("Poisson 2000 requests/s (trace seed 5), first %d requests replayed at their arrival "
                       "times" % args.serve_requests)
    bounded = [r["offered_req_per_s"] for r in sweep if r["failed"] == 0 and r["p99_ms"] <= 4 * max(
        sweep[0]["p99_ms"], 1.0)]
    return {"sweep": sweep, "overload_2000_req_s": over,
            "p99_bounded_up_to_req_s": max(bounded) if bounded else None,
            "mix": "n log-uniform [64, 16384]; half fp32->fp64, half fp64->double-double; half all pairs, half "
                   "10% index ranges; host inputs, device outputs; 3 workers, budget = half the free HBM",
            "bounded_rule": "p99 within 4x of the p99 at the lowest offered rate"}


def _e2e(m, mats_h, args, dev):
    """The C2 step end to end through the C ABI with host buffers: one
    mrrr_solve_batch_s call given pinned host pointers for d, e, W and Z (ldz
    = n); the library copies the inputs to the device, solves, and copies W
    and Z back before it returns, all inside the timed region (wall clock)."""
    import ctypes
    import torch
    nb = len(mats_h)
    n = [d.size for d, _ in mats_h]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    dh = [pin(d) for d, _ in mats_h]
    eh = [pin(e) for _, e in mats_h]
    Wh = [torch.empty(k, dtype=torch.float32).pin_memory() for k in n]
    Zh = [torch.empty((k, k), dtype=torch.float32).pin_memory() for k in n]
    vp = ctypes.c_void_p

    def arr(t, xs):
        return ctypes.cast((t * nb)(*xs), vp)

    a_n = arr(ctypes.c_int, n)
    a_d = arr(vp, [t.data_ptr() for t in dh])
    a_e = arr(vp, [t.data_ptr() for t in eh])
    a_w = arr(vp, [t.data_ptr() for t in Wh])
    a_z = arr(vp, [t.data_ptr() for t in Zh])
    a_ld = arr(ctypes.c_int, n)
    status = (ctypes.c_int * nb)()
    mout = (ctypes.c_int * nb)()
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def step():
        rc = m.mrrr_solve_batch_s(nb, a_n, a_d, a_e, None, None, m.MRRR_MIXED, None, ctypes.cast(mout, vp), a_w,
                                  a_z, a_ld, ctypes.cast(status, vp), stream)
        assert rc == 0, rc

    for _ in range(max(1, args.warmup)):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    pairs = sum(n)
    h2d = sum(4 * (d.size + e.size) for d, e in mats_h)
    d2h = sum(4 * (k + k * k) for k in n)
    return {"value": pairs * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "api": "mrrr_solve_batch_s with pinned host buffers for d, e, W and Z: the library stages them "
                   "through device memory inside the call; wall clock per call"}


def _spawn(args):
    """--gpus N outside a distributed launcher: start N ranks on this node
    through torch.distributed.run (one process per GPU) and return its status."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(args.gpus),
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched, C3, C4 and serving measurements")
    ap.add_argument("--step-only", action="store_true",
                    help="only the warm-up and timed steps of the headline workload (for profiling)")
    ap.add_argument("--extra-steps", type=int, default=10, help="timed steps of the C3 and C4 legs")
    ap.add_argument("--serve-rates", type=float, nargs="*", default=[2.0, 5.0, 10.0, 20.0],
                    help="offered Poisson rates (requests/s) of the serving sweep")
    ap.add_argument("--serve-seconds", type=float, default=6.0, help="arrival window of each sweep point")
    ap.add_argument("--serve-requests", type=int, default=200, help="requests replayed from the 2000/s trace")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if "WORLD_SIZE" in os.environ and world != args.gpus:
        sys.stderr.write("bench.py: --gpus %d but WORLD_SIZE=%d\n" % (args.gpus, world))
        return 2
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return _spawn(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
