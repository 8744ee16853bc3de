"""Benchmark: batched exact metric range / kNN search over a GTS index on GB300.

Headline workload (one JSON line, rank 0): 1,000,000 float32 vectors of dim
128 from a mixture of 64 isotropic Gaussians (centres uniform in [-1, 1],
sigma 0.1, seed 0); 10,000 kNN queries, k = 10, from the same mixture (seed
1); node capacity 20, h = 4 (Algorithm 1).  One step = one gts_knn call over
the whole 10,000-query batch: pivot distances, node pruning, the kNN
threshold, the list-table bound, verification and selection, all on the GPU.

* `value`: queries/s over all ranks with the index and queries resident in
  HBM, timed over K steps with no per-stage instrumentation.
* `e2e`: the same metric through the C ABI with pinned host queries and host
  results (copies inside the timed region).
* `stage_ms_per_step` and `roofline`: a second pass of K steps with CUDA
  events around every launch of each stage (on the query stream), plus one
  untimed call that counts the (query, row) pairs passing the table lower
  bound (C_q); the tile stage's algorithmic work is 2 D C_q flops.
* `other_workloads` (single-GPU runs): the other configurations, each
  timed on its own with its build and rebuild times -- words_10k_r2 and
  dna_1M_r8 (edit distance, range), zipf2d_10M (10^7 2-D points, range
  queries with stream inserts / deletes and a batch update inside the timed
  region), wordvec_200kx300_cos (angular-distance kNN over 200,000
  word-vector-like rows of dim 300), uniform_2Mx256_l1 (served Poisson
  arrivals, p50 / p99).

The index (X 512 MB, table 16 MB) is larger than L2 (129 MB), so no explicit
flush runs between steps.

--impl reference: the CPU oracle (brute force, FP64, all host cores) on a
bounded sample of the same queries per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
import traceback

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
SMS = 152                     # GB300: 152 SMs
FP32_LANES_PER_SM = 128       # FP32 FMA lanes per SM
ALU_LANES_PER_SM = 64         # integer / bit-logic ALU pipe: 2 warp instructions per SM cycle (ncu: the ALU
                              # instructions executed per active SM cycle are exactly 2 x its pipe utilization)

# DRAM bytes per launch of the dominant kernel from one ncu capture (profiles/):
# k_tile_l2_tc at half size, 0.467 GB read + write (node rows, the node x
# query leaf-mask matrix and the kept pairs' q.x), all of which double at full
# size.  None once the kernel has changed since the counters were taken.
TRAFFIC = {"kernel": "tile", "bytes_per_launch": 0.934e9}
# the zipf2d table scan (k_scan_warps, fused range form): DRAM read + write of
# one launch over a 10,000-query batch from its ncu capture
# (profiles/scan_warps_zipf2d_10M.md), 227.1 + 101.6 MB.  None once the kernel
# changes.
SCAN_TRAFFIC = 328.7e6

# ALU-pipe thread instructions per full-DP-equivalent cell (|q| x |o| per pair)
# of the bit-parallel edit-distance kernels: sm__inst_executed_pipe_alu.sum x 32
# over the cells of every launch of one batch pair of the dna workload at 0.2
# scale (profiles/dp_str_dna_200k_r8.md).  None once the kernels change.
INT_OPS_PER_CELL = {"pivot_dist": 0.600, "verify": 0.619}


def workload(scale: float = 1.0):
    from synth import gaussian_mixture
    n = int(1_000_000 * scale)
    nq = max(64, int(10_000 * scale))
    cache = os.path.join(os.environ.get("GTS_SYNTH_CACHE", "/tmp/gts_synth_cache"), f"gauss_{n}_{nq}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        return z["X"], z["Q"], int(z["k"])
    wl = gaussian_mixture(n=n, dim=128, n_centers=64, sigma=0.1, nq=nq, k=10)
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    try:
        np.savez(cache, X=wl.objects, Q=wl.queries, k=10)
    except OSError:
        pass
    return wl.objects, wl.queries, 10


def _measured():
    try:
        with open(MEASURED) as f:
            return json.load(f)
    except Exception:
        return None


def peaks():
    m = _measured()
    return (float(m["hbm_gbs"]), "measured") if m else (FALLBACK_HBM_GBS, "fallback")


def tensor_peak():
    """Sustained dense bf16 TFLOP/s (a kernel timed inside a long step)."""
    m = _measured()
    return (float(m["bf16_tflops_sustained"]), "measured") if m else (1700.0, "fallback")


def alu_peak(sm_mhz, lanes=ALU_LANES_PER_SM):
    """Lane-operation peak (T thread-instructions/s) of a pipe from the unit
    counts: 152 SMs x its lanes per SM x the SM clock (the median sampled
    under load, else the maximum 2070 MHz)."""
    mhz = sm_mhz or 2070.0
    return SMS * lanes * mhz * 1e6 / 1e12, mhz


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
            f = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(X, Q, k, budget_s=12.0):
    """The oracle as it stands (brute force, FP64) on a bounded sample of the
    same queries, all host cores."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.knn_query("l2", X, Q[:8], k)
    per_q = (time.perf_counter() - t0) / 8
    m = int(max(8, min(Q.shape[0], budget_s / max(per_q, 1e-6))))
    t0 = time.perf_counter()
    oracle.knn_query("l2", X, Q[8:8 + m] if 8 + m <= Q.shape[0] else Q[:m], k)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": "queries/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"{m} of the {Q.shape[0]} queries, full 1M x 128 dataset, brute-force FP64 kNN (k={k})"}


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def stage_pass(step, steps, stream):
    """K more steps with per-stage CUDA events: device ms per stage and step,
    launches per stage and step, and the first step's counters."""
    import torch
    stage_ms, stage_launch, stats0 = {}, {}, None
    torch.cuda.synchronize()
    for _ in range(steps):
        st = step(timing=True)
        stats0 = stats0 or st
        for kk, v in st["stage_ms"].items():
            stage_ms[kk] = stage_ms.get(kk, 0.0) + v / steps
        for kk, v in st["stage_launches"].items():
            stage_launch[kk] = stage_launch.get(kk, 0) + v / steps
    torch.cuda.synchronize()
    return stage_ms, stage_launch, stats0


def run_ours(args):
    import torch
    import paper_2404_00966_gb300 as gts
    from paper_2404_00966_gb300 import build_ext

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build_ext.build()
    if dist:
        dist.barrier()
    X, Q, k = workload(args.scale)
    nq, dim = Q.shape
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    Kd = torch.full((nq,), k, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gts.Index.build(Xd, "l2", fanout=20, root_pivot=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    info = ix.info()
    prec = args.precision
    stream = torch.cuda.current_stream()
    # launch parameters for this index and batch shape (gts_autotune; untimed
    # setup like the build; every setting returns the same answers)
    tuning = ix.autotune(Qd, k=np.full(nq, k, np.int32), precision=prec, reps=2) if not args.no_tune else None

    def step_prec(p, timing=False, count=False):
        r = ix.knn(Qd, Kd, precision=p, result_on_device=True, timing=timing, count_table_pass=count)
        st = r.stats
        r.free()
        return st

    def step(timing=False):
        return step_prec(prec, timing)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # ---- timed region: device-resident inputs, no per-stage instrumentation
    launches = 0
    stats0 = None
    with ClockSampler(local) as clocks:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        e0.record(stream)
        marks[0].record(stream)
        for i in range(args.steps):
            st = step()
            marks[i + 1].record(stream)
            stats0 = stats0 or st
            launches += st["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    per_batch = np.array([marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps)])
    ms_step = ms / args.steps
    value = world * nq * args.steps / (ms / 1e3)
    # ---- end to end: pinned host queries, host results
    Qh = torch.from_numpy(Q).pin_memory()
    Kh = torch.full((nq,), k, dtype=torch.int32).pin_memory()
    ix.knn(Qh, Kh, precision=prec)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    tot_res = 0
    for _ in range(args.steps):
        r = ix.knn(Qh, Kh, precision=prec)
        tot_res = int(r.offsets[-1])
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": world * nq * args.steps / e2e_s, "unit": "queries/s",
           "h2d_bytes_per_step": int(Qh.numel() * 4 + Kh.numel() * 4),
           "d2h_bytes_per_step": int((nq + 1) * 8 + tot_res * 12)}
    # ---- stage breakdown: K more steps with CUDA events around every launch
    stage_ms, stage_launch, _ = stage_pass(step, args.steps, stream)
    # the (query, row) pairs passing the table lower bound (untimed call)
    cq = step_prec(prec, count=True)["table_pass"]
    # ---- roofline of the dominant stage
    dom = max(stage_ms, key=lambda s_: stage_ms[s_])
    dom_ms = stage_ms[dom]
    hbm, src = peaks()
    if dom == "tile" and prec == "bf16":
        # a contraction on the tensor cores: the algorithm's work is 2 D flops
        # per (query, row) pair that passes the table lower bound (C_q), against
        # the sustained bf16 peak (the kernel runs inside a long step).  The
        # tiles compute every row of a surviving node block (covered pairs),
        # and the split-bf16 form executes 3 products per pair.
        tf, tsrc = tensor_peak()
        sec = dom_ms / 1e3
        achieved = cq * 2 * dim / sec / 1e12 if dom_ms > 0 else 0.0
        covered = stats0["tile_pairs"] * 2 * dim / sec / 1e12 if dom_ms > 0 else 0.0
        roof = {"bound": "tensor", "kernel": "k_tile_l2_tc (stage tile)", "achieved": round(achieved, 2), "peak": tf,
                "unit": "TFLOP/s", "frac": round(achieved / tf, 5), "peak_source": tsrc,
                "traffic": TRAFFIC["bytes_per_launch"] if TRAFFIC["kernel"] == dom else None,
                "launches_per_step": stage_launch[dom], "ms_per_step": round(dom_ms, 4),
                "algorithmic_pairs_per_step": int(cq),
                "covered_pairs_per_step": int(stats0["tile_pairs"]),
                "covered_tflops": round(covered, 1), "covered_frac": round(covered / tf, 4),
                "executed_tflops": round(3 * covered, 1), "executed_frac": round(3 * covered / tf, 4)}
    else:
        roof = {"bound": "latency", "kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": None, "launches_per_step": stage_launch[dom], "ms_per_step": round(dom_ms, 4)}
    counters = {kk: v for kk, v in stats0.items() if not isinstance(v, dict)}
    counters["table_pass"] = int(cq)
    out = {
        "metric": "kNN queries/s at oracle-exact results (L2, k=10)",
        "value": round(value, 1), "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f64" if prec == "bf16" else "f32+f64", "data": "synthetic",
        "config": {"workload": "gauss64_1Mx128_knn10", "n": int(X.shape[0]), "dim": int(dim), "nq": int(nq),
                   "k": k, "fanout": 20, "h": info["h"], "precision": prec,
                   "l2_flush": "inputs larger than L2 (vectors 512 MB + table 16 MB per step)",
                   "parallelism": f"replicas{world}", "build_s": round(build_s, 3), "tuning": tuning},
        "e2e": {kk: (round(v, 1) if isinstance(v, float) else v) for kk, v in e2e.items()},
        # every query of a batch completes with its batch: per-query latency = the batch's time
        "latency_ms": {"p50": round(float(np.percentile(per_batch, 50)), 3),
                       "p99": round(float(np.percentile(per_batch, 99)), 3),
                       "of": f"one {nq}-query batch (device inputs)"},
        "gpu_launches": int(launches),
        "roofline": roof,
        "stage_ms_per_step": {kk: round(v, 4) for kk, v in stage_ms.items()},
        "stage_timing": "a second pass of the same steps with CUDA events around every launch",
        "counters_per_step": counters,
        "clocks": clocks.summary(),
    }
    if prec == "bf16" and not args.no_fp32_compare:
        # the plain FP32 single-batch path on the same index and queries
        step_prec("fp32")
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nfs = max(1, min(3, args.steps))
        f0.record(stream)
        for _ in range(nfs):
            step_prec("fp32")
        f1.record(stream)
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1) / nfs
        out["fp32_plain"] = {"value": round(world * nq / (fms / 1e3), 1), "unit": "queries/s",
                             "ms_per_step": round(fms, 3), "steps": nfs}
    ix.close()
    del Xd, Qd
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(X, Q, k, budget_s=args.cpu_seconds)
    if rank == 0 and world == 1 and not args.no_others:
        out["other_workloads"] = run_others(args)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other workloads (also parity-test configurations)

def _dev_strings(S):
    import torch
    return (torch.from_numpy(S.data if S.data.size else np.zeros(1, np.uint8)).cuda(),
            torch.from_numpy(S.offsets).cuda())


def calibrate_radius(ix, cal, target, torch, iters=24):
    """Radius whose mean range-result count over the calibration queries is
    about `target` (bisection in log space)."""
    ncal = cal.shape[0]
    rk = ix.knn(cal, int(min(target, 1024)))
    hi = float(np.max([rk.query(i)[1][-1] for i in range(ncal)])) * 4.0
    lo = hi / 1e6
    for _ in range(iters):
        mid = (lo * hi) ** 0.5
        res = ix.range(cal, torch.full((ncal,), mid, dtype=torch.float32, device="cuda"))
        mean = float(res.offsets[-1]) / ncal
        if mean > target:
            hi = mid
        else:
            lo = mid
        if abs(mean - target) < 0.02 * target:
            return mid
    return (lo * hi) ** 0.5


def _timed_steps(step, steps, warmup, stream, local):
    """Warm-up, then K steps between CUDA events; per-step stats of the first."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    launches, stats0 = 0, None
    with ClockSampler(local) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            st = step()
            stats0 = stats0 or st
            launches += st["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1), launches, stats0, clocks.summary()


def bench_strings(name, args):
    """words_10k_r2 or dna_1M_r8: edit-distance range queries, exact int32."""
    import torch
    import paper_2404_00966_gb300 as gts
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    stream = torch.cuda.current_stream()
    prec = args.precision
    if name == "words":
        wl = synth.words_like()
    else:   # --scale < 1: fewer seeds and queries (profiling only)
        wl = synth.dna_like() if args.scale >= 1.0 else synth.dna_like(
            n_seeds=max(100, int(10_000 * args.scale)), nq=max(100, int(20_000 * args.scale)))
    objs = _dev_strings(wl.objects)
    queries = _dev_strings(wl.queries)
    radii = torch.from_numpy(wl.radii).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gts.Index.build(objs, "edit", n_pivots=wl.n_pivots, fanout=wl.fanout, root_pivot=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix.rebuild()
    torch.cuda.synchronize()
    rebuild_s = time.perf_counter() - t0
    nq = wl.nq

    def step(timing=False):
        r = ix.range(queries, radii, precision=prec, result_on_device=True, timing=timing)
        st = r.stats
        r.free()
        return st
    ms, launches, stats0, clocks = _timed_steps(step, args.other_steps, args.warmup, stream, local)
    stage_ms, stage_launch, _ = stage_pass(step, args.other_steps, stream)
    out = {"metric": f"range queries/s at oracle-exact results (edit, r={int(wl.radii[0])})",
           "value": round(nq * args.other_steps / (ms / 1e3), 1), "unit": "queries/s", "steps": args.other_steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.other_steps, 4), "dtype": "int32",
           "config": {"workload": wl.name, "n": int(wl.objects.n), "nq": nq, "fanout": wl.fanout,
                      "h": ix.info()["h"], "precision": prec},
           "build_s": round(build_s, 3), "rebuild_s": round(rebuild_s, 3),
           "gpu_launches": int(launches), "stage_ms_per_step": {kk: round(v, 4) for kk, v in stage_ms.items()},
           "counters_per_step": {kk: v for kk, v in stats0.items() if not isinstance(v, dict)}, "clocks": clocks}
    # edit distance: DP cells (full-matrix equivalent) per second of the two DP
    # stages; INT32 roofline from the integer / bit-logic instructions per cell
    # (ncu) against the lane peak
    lq = float(np.mean(np.diff(wl.queries.offsets)))
    lo = float(np.mean(np.diff(wl.objects.offsets)))
    rates = {}
    for stage, pairs in (("pivot_dist", stats0["pivot_dist"]), ("verify", stats0["candidates"])):
        sec = stage_ms.get(stage, 0.0) / 1e3
        if sec > 0:
            rates[stage] = pairs * lq * lo / sec
    dom = max(stage_ms, key=lambda s_: stage_ms[s_])
    peak, mhz = alu_peak(clocks.get("sm_mhz"))
    if dom in rates and INT_OPS_PER_CELL.get(dom):
        ach = rates[dom] * INT_OPS_PER_CELL[dom] / 1e12
        out["roofline"] = {"bound": "alu", "kernel": dom, "unit": "T ALU-pipe thread instructions/s",
                           "achieved": round(ach, 3), "peak": round(peak, 2), "frac": round(ach / peak, 4),
                           "peak_source": f"{SMS} SMs x {ALU_LANES_PER_SM} ALU lanes x {mhz:.0f} MHz (derived)",
                           "int_ops_per_cell": INT_OPS_PER_CELL[dom],
                           "dp_cells_per_s": {kk: round(v, 1) for kk, v in rates.items()}, "traffic": None}
    else:
        out["roofline"] = {"bound": "latency" if name == "words" else "alu", "kernel": dom, "achieved": None,
                           "peak": None, "frac": None,
                           "dp_cells_per_s": {kk: round(v, 1) for kk, v in rates.items()}, "traffic": None}
    ix.close()
    if not args.no_cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.range_query("edit", wl.objects, wl.queries.take(np.arange(2)), wl.radii[:2])
        per_q = (time.perf_counter() - t0) / 2
        m = int(max(2, min(nq, args.other_cpu_seconds / max(per_q, 1e-6))))
        t0 = time.perf_counter()
        oracle.range_query("edit", wl.objects, wl.queries.take(np.arange(m)), wl.radii[:m])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(m / dt, 3), "unit": "queries/s", "cores": oracle.threads(),
                               "kind": "oracle", "sample": f"{m} queries, brute-force banded edit distance"}
    return out


def bench_zipf2d(args):
    """zipf2d_10M: 10^7 2-D points, L2 range queries at ~0.01% selectivity.
    One step = a 10,000-query batch followed by 500 stream inserts and 500
    stream deletes (10% updates); the step after the fifth also runs the
    batch update (rebuild with 500,000 more points).  Ten steps = the
    workload's 100,000 queries, updates inside the timed region."""
    import torch
    import paper_2404_00966_gb300 as gts
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    stream = torch.cuda.current_stream()
    prec = args.precision
    wl = synth.zipf_clusters_2d(nq=100_000)
    Xd = torch.from_numpy(wl.objects).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gts.Index.build(Xd, "l2", fanout=20, root_pivot=0, cache_limit=4096)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix.rebuild()
    torch.cuda.synchronize()
    rebuild_s = time.perf_counter() - t0
    del Xd
    # one global radius with a mean result count of ~1,000 (0.01%) over 1,000
    # calibration queries: bisection on the range-query counts
    cal = torch.from_numpy(wl.queries[:1000]).cuda()
    r = calibrate_radius(ix, cal, 1000.0, torch)
    nb = 10_000
    Qall = torch.from_numpy(wl.queries).cuda()
    radii = torch.full((nb,), r, dtype=torch.float32, device="cuda")
    upd = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 10_000, seed=2)
    bulk = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 500_000, seed=5)
    drng = np.random.default_rng(3)
    qa, qz = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    state = {"round": 0, "timed": False, "q_ms": 0.0, "u_s": 0.0, "bu_s": 0.0}

    def queries_only(timing=False):
        res = ix.range(Qall[:nb], radii, precision=prec, result_on_device=True, timing=timing)
        st = res.stats
        res.free()
        return st

    def step():
        i = state["round"]
        qb = Qall[(i % 10) * nb:((i % 10) + 1) * nb]
        qa.record(stream)
        res = ix.range(qb, radii, precision=prec, result_on_device=True)
        qz.record(stream)
        st = res.stats
        res.free()
        u0 = time.perf_counter()
        ix.insert(upd[(i * 500) % 9_500:(i * 500) % 9_500 + 500])
        info = ix.info()
        ix.delete(drng.integers(0, info["next_id"], size=500))
        torch.cuda.synchronize()
        u1 = time.perf_counter()
        if i == 5:
            ix.batch_update(bulk)   # one batch update: rebuild with 500,000 more points
            torch.cuda.synchronize()
        u2 = time.perf_counter()
        if state["timed"]:
            state["q_ms"] += qa.elapsed_time(qz)   # both recorded before the synchronize above
            state["u_s"] += u1 - u0
            state["bu_s"] += u2 - u1
        state["round"] += 1
        return st
    for _ in range(args.warmup):
        queries_only()
    torch.cuda.synchronize()
    state["timed"] = True
    launches, stats0 = 0, None
    with ClockSampler(local) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            st = step()
            stats0 = stats0 or st
            launches += st["launches"]
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stage_ms, stage_launch, st1 = stage_pass(queries_only, args.other_steps, stream)
    # the node-major table scan (stage leaf_scan): bytes it must move per launch
    # = every staged row once (h table columns, its delete mark, its 2-D point)
    # + every (query, row block) record with its path distances + the answers
    # and band pairs it writes; against the measured HBM copy peak
    info = ix.info()
    h = info["h"]
    hbm, hsrc = peaks()
    scan_ms = stage_ms.get("leaf_scan", 0.0)
    scan_bytes = (st1["scanned_rows"] * (4 * h + 8 + 4 * 2) + st1["scan_records"] * (32 + 4 * ((h + 3) // 4 * 4))
                  + st1["results"] * 12)
    scan_roof = None
    if scan_ms > 0:
        gbs = scan_bytes / (scan_ms / 1e3) / 1e9
        scan_roof = {"bound": "hbm", "kernel": "k_scan_warps (stage leaf_scan)", "achieved": round(gbs, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(gbs / hbm, 4), "peak_source": hsrc,
                     "bytes_per_launch": int(scan_bytes),
                     "ms_per_launch": round(scan_ms / max(1.0, stage_launch.get("leaf_scan", 1.0)), 4),
                     "traffic": SCAN_TRAFFIC}
    out = {"metric": "range queries/s at oracle-exact results (L2, ~0.01% selectivity, 10% stream updates "
                     "and a 500,000-point batch update inside the timed region)",
           "value": round(10 * nb / (ms / 1e3), 1), "unit": "queries/s", "steps": 10, "warmup": args.warmup,
           "ms_per_step": round(ms / 10, 4), "dtype": "bf16+f64" if prec == "bf16" else "f32+f64",
           "config": {"workload": "zipf2d_10M", "n": 10_000_000, "nq": 10 * nb, "radius": r, "fanout": 20,
                      "h": ix.info()["h"], "precision": prec},
           "query_only": {"value": round(10 * nb / (state["q_ms"] / 1e3), 1), "unit": "queries/s",
                          "ms_per_step": round(state["q_ms"] / 10, 4)},
           "update_ms_per_step": round(1e3 * state["u_s"] / 10, 3),
           "batch_update_s": round(state["bu_s"], 3),
           "build_s": round(build_s, 3), "rebuild_s": round(rebuild_s, 3),
           "gpu_launches": int(launches), "roofline": scan_roof,
           "stage_ms_per_step": {kk: round(v, 4) for kk, v in stage_ms.items()},
           "counters_per_step": {kk: v for kk, v in stats0.items() if not isinstance(v, dict)},
           "clocks": clocks.summary()}
    ix.close()
    return out


def bench_serving(args):
    """uniform_2Mx256_l1: 2,000,000 x 256 uniform vectors, L1; requests arrive
    as a Poisson stream at 50,000/s (half range queries with a radius of ~100
    results, half kNN with k uniform in 1..100) and are served by the
    continuous-batching loop under a 16 GB admission budget.  Served
    requests/s and the p50 / p99 latency from submit to result."""
    import torch
    import paper_2404_00966_gb300 as gts
    import synth
    nreq = args.requests
    wl = synth.uniform_cube(n=2_000_000, dim=256, nq=nreq + 512)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gts.Index.build(torch.from_numpy(wl.objects).cuda(), "l1", fanout=20, root_pivot=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    cal = torch.from_numpy(wl.queries[nreq:nreq + 256]).cuda()
    radius = calibrate_radius(ix, cal, 100.0, torch, iters=16)
    is_knn, ks = synth.mixed_requests(nreq, seed=1)
    arrivals = synth.poisson_arrivals(nreq, args.rate, seed=1)
    sv = gts.Server(ix, max_batch=args.max_batch, n_streams=args.serve_streams, precision=args.precision,
                    result_budget=16 << 30, batch_quantum=args.batch_quantum)
    warm = [sv.submit(wl.queries[nreq + i], "knn", 10) for i in range(64)]
    for t in warm:
        sv.wait(t)
    tickets = []
    sub_t = np.zeros(nreq)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        start = time.perf_counter()
        for i in range(nreq):
            target = start + arrivals[i]
            while True:
                now = time.perf_counter()
                if now >= target:
                    break
                if target - now > 2e-3:
                    time.sleep(target - now - 1e-3)
            sub_t[i] = time.perf_counter() - start
            tickets.append(sv.submit(wl.queries[i], "knn" if is_knn[i] else "range",
                                     int(ks[i]) if is_knn[i] else radius))
        lat = np.zeros(nreq)
        for i, t in enumerate(tickets):
            lat[i] = sv.wait(t)[2]
    st = sv.stats()
    sv.stop()
    done_t = sub_t + lat / 1e3
    span = float(done_t.max())
    out = {"metric": "served mixed range/kNN requests/s (L1, Poisson arrivals, 16 GB admission budget); p50/p99 ms",
           "value": round(nreq / span, 1), "unit": "requests/s", "steps": 1, "warmup": 1,
           "ms_per_step": round(1e3 * span, 2), "dtype": "f32+f64",
           "config": {"workload": "uniform_2Mx256_l1_serving", "n": 2_000_000, "dim": 256, "requests": nreq,
                      "arrival_rate": args.rate, "radius": radius, "max_batch": args.max_batch,
                      "streams": args.serve_streams, "batch_quantum": args.batch_quantum,
                      "precision": args.precision},
           "build_s": round(build_s, 3),
           "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                          "mean": round(float(lat.mean()), 3), "max": round(float(lat.max()), 3)},
           "offered_span_s": round(float(arrivals[-1]), 4), "server": st,
           "admission": {"projected_bytes_per_request": round(st["projected_bytes"] / max(1, st["requests"]), 1),
                         "worst_case_bytes_per_request": 2_000_000 * 37,
                         "requests_below_worst_case": st["below_worst_case"],
                         "result_budget_bytes": 16 << 30},
           "clocks": clocks.summary()}
    ix.close()
    return out


def bench_wordvec(args):
    """wordvec_200000x300_cos_knn10: angular-distance kNN over word-vector-like
    data (the Vector data's shape), BF16 tiles on the unit vectors and the
    FP64 key 1 - cos of every answer."""
    import torch
    import paper_2404_00966_gb300 as gts
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    stream = torch.cuda.current_stream()
    prec = args.precision
    wl = synth.word_vectors() if args.scale >= 1.0 else synth.word_vectors(n=max(20_000, int(200_000 * args.scale)))
    X, Q, k = wl.objects, wl.queries, int(wl.k[0])
    nq, dim = Q.shape
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    Kd = torch.from_numpy(wl.k).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ix = gts.Index.build(Xd, "cos", fanout=wl.fanout, root_pivot=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    ix.rebuild()
    torch.cuda.synchronize()
    rebuild_s = time.perf_counter() - t0
    # untimed setup like the build: the index shape by the cost model and a
    # timed sample batch (pruning is weak on these 300-dimensional directions,
    # so shallower trees with larger node blocks win), then launch parameters
    shapes = ix.autotune_shape(Qd[:2000], k=10, precision=prec, candidates=4, reps=1) if not args.no_tune else None
    tuning = ix.autotune(Qd, k=wl.k, precision=prec, reps=2) if not args.no_tune else None

    def step(timing=False, count=False):
        r = ix.knn(Qd, Kd, precision=prec, result_on_device=True, timing=timing, count_table_pass=count)
        st = r.stats
        r.free()
        return st
    ms, launches, stats0, clocks = _timed_steps(step, args.other_steps, args.warmup, stream, local)
    stage_ms, stage_launch, _ = stage_pass(step, args.other_steps, stream)
    cq = step(count=True)["table_pass"]
    dom = max(stage_ms, key=lambda s_: stage_ms[s_])
    out = {"metric": "kNN queries/s at oracle-exact results (angular distance, k=10)",
           "value": round(nq * args.other_steps / (ms / 1e3), 1), "unit": "queries/s", "steps": args.other_steps,
           "warmup": args.warmup, "ms_per_step": round(ms / args.other_steps, 4),
           "dtype": "bf16+f64" if prec == "bf16" else "f32+f64",
           "config": {"workload": wl.name, "n": int(X.shape[0]), "dim": int(dim), "nq": int(nq), "k": k,
                      "fanout": ix.info()["fanout"], "h": ix.info()["h"], "precision": prec, "tuning": tuning,
                      "shapes_timed": shapes},
           "build_s": round(build_s, 3), "rebuild_s": round(rebuild_s, 3),
           "gpu_launches": int(launches), "stage_ms_per_step": {kk: round(v, 4) for kk, v in stage_ms.items()},
           "counters_per_step": {**{kk: v for kk, v in stats0.items() if not isinstance(v, dict)},
                                 "table_pass": int(cq)},
           "clocks": clocks}
    if dom == "tile" and prec == "bf16" and stage_ms[dom] > 0:
        tf, tsrc = tensor_peak()
        sec = stage_ms[dom] / 1e3
        ach = cq * 2 * dim / sec / 1e12
        cov = stats0["tile_pairs"] * 2 * dim / sec / 1e12
        out["roofline"] = {"bound": "tensor", "kernel": "k_tile_l2_tc (stage tile)", "achieved": round(ach, 2),
                           "peak": tf, "unit": "TFLOP/s", "frac": round(ach / tf, 5), "peak_source": tsrc,
                           "traffic": None, "ms_per_step": round(stage_ms[dom], 4),
                           "covered_tflops": round(cov, 1), "executed_tflops": round(3 * cov, 1)}
    else:
        out["roofline"] = {"bound": "latency", "kernel": dom, "achieved": None, "peak": None, "frac": None,
                           "traffic": None, "ms_per_step": round(stage_ms[dom], 4)}
    ix.close()
    del Xd, Qd
    if not args.no_cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.knn_query("cos", X, Q[:8], 10)
        per_q = (time.perf_counter() - t0) / 8
        m = int(max(8, min(nq, args.other_cpu_seconds / max(per_q, 1e-6))))
        t0 = time.perf_counter()
        oracle.knn_query("cos", X, Q[:m], 10)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(m / dt, 3), "unit": "queries/s", "cores": oracle.threads(),
                               "kind": "oracle", "sample": f"{m} queries, brute-force FP64 angular kNN"}
    return out


def bench_multicol(args):
    """multicol_200000_l2x128_cos300_knn10: multi-column kNN over an L2
    column and an angular column of one object set (distance = the sum of
    the two), through gts_multi_knn: host queries in, host answers out, the
    threshold algorithm's rounds and random accesses inside the timed call."""
    import torch
    import paper_2404_00966_gb300 as gts
    import synth
    local = int(os.environ.get("LOCAL_RANK", "0"))
    prec = args.precision
    wl = synth.multi_columns() if args.scale >= 1.0 else synth.multi_columns(n=max(20_000, int(200_000 * args.scale)))
    nq, k = int(wl.queries[0].shape[0]), int(wl.k[0])
    cols, shapes = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for X, m in zip(wl.objects, wl.metrics):
        cols.append(gts.Index.build(torch.from_numpy(X).cuda(), m, fanout=wl.fanout, root_pivot=0))
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    if not args.no_tune:   # untimed setup: each column's shape by the cost model and a sample batch
        for ix, Q in zip(cols, wl.queries):
            shapes.append(ix.autotune_shape(torch.from_numpy(Q[:2000]).cuda(), k=k, precision=prec, candidates=4,
                                            reps=1))

    def step():
        return gts.multi_knn(cols, wl.queries, wl.k, precision=prec)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches = 0
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for _ in range(args.other_steps):
            r = step()
            launches += r.stats["launches"]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    out = {"metric": "multi-column kNN queries/s at oracle-exact results (L2 + angle, k=10)",
           "value": round(nq * args.other_steps / dt, 1), "unit": "queries/s", "steps": args.other_steps,
           "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.other_steps, 3),
           "dtype": "bf16+f64" if prec == "bf16" else "f32+f64", "timing": "host wall clock around the call",
           "config": {"workload": wl.name, "n": int(wl.objects[0].shape[0]), "columns": wl.metrics,
                      "dims": [int(x.shape[1]) for x in wl.objects], "nq": nq, "k": k, "precision": prec,
                      "shapes": shapes},
           "answers": int(r.offsets[-1]), "build_s": round(build_s, 3), "gpu_launches": int(launches),
           "counters_per_step": r.stats, "clocks": clocks.summary()}
    for ix in cols:
        ix.close()
    if not args.no_cpu:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.multi_knn(wl.metrics, wl.objects, [q[:2] for q in wl.queries], k)
        per_q = (time.perf_counter() - t0) / 2
        m = int(max(2, min(nq, args.other_cpu_seconds / max(per_q, 1e-6))))
        t0 = time.perf_counter()
        oracle.multi_knn(wl.metrics, wl.objects, [q[:m] for q in wl.queries], k)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(m / dt, 3), "unit": "queries/s", "cores": oracle.threads(),
                               "kind": "oracle", "sample": f"{m} queries, brute-force FP64 summed distances"}
    return out


def run_others(args):
    """Each remaining configuration timed on its own; a failure is recorded
    in its entry and does not stop the others."""
    import torch
    out = {}
    for name, fn in (("words_10k_r2", lambda: bench_strings("words", args)),
                     ("dna_1M_r8", lambda: bench_strings("dna", args)),
                     ("zipf2d_10M", lambda: bench_zipf2d(args)),
                     ("wordvec_200kx300_cos", lambda: bench_wordvec(args)),
                     ("multicol_200k_l2x128_cos300", lambda: bench_multicol(args)),
                     ("uniform_2Mx256_l1_serving", lambda: bench_serving(args))):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:   # keep the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}", "trace": traceback.format_exc()[-800:]}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()
    return out


def run_config(args):
    """One of the other workloads alone (--workload words|dna|zipf2d|wordvec|multicol|serving)."""
    import torch
    from paper_2404_00966_gb300 import build_ext
    build_ext.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    if args.workload in ("words", "dna"):
        out = bench_strings(args.workload, args)
    elif args.workload == "zipf2d":
        out = bench_zipf2d(args)
    elif args.workload == "wordvec":
        out = bench_wordvec(args)
    elif args.workload == "multicol":
        out = bench_multicol(args)
    else:
        out = bench_serving(args)
    out.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic"})
    print(json.dumps(out), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    X, Q, k = workload(args.scale)
    m = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        sl = Q[(i * m) % Q.shape[0]:(i * m) % Q.shape[0] + m]
        t0 = time.perf_counter()
        oracle.knn_query("l2", X, sl, k)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    tot = sum(times)
    value = m * len(times) / tot
    sample = f"{m} queries per step of the {Q.shape[0]}, full 1M x 128 dataset, brute-force FP64 kNN (k={k})"
    out = {"impl": "reference", "metric": "kNN queries/s at oracle-exact results (L2, k=10)",
           "value": round(value, 3), "unit": "queries/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot / len(times), 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "gauss64_1Mx128_knn10", "n": int(X.shape[0]), "dim": 128, "nq": int(Q.shape[0]),
                      "k": k},
           "cpu_baseline": {"value": round(value, 3), "unit": "queries/s", "cores": oracle.threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 3), "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload (profiling only)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the default launch parameters")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-sample", type=int, default=32)
    ap.add_argument("--requests", type=int, default=20_000, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=50_000.0, help="serving: mean arrivals per second")
    ap.add_argument("--max-batch", type=int, default=1024, help="serving: requests per device batch")
    ap.add_argument("--serve-streams", type=int, default=2, help="serving: worker streams (batches in flight)")
    ap.add_argument("--batch-quantum", type=int, default=64,
                    help="serving: cut batches down to a multiple of this many requests (0 = no rounding); "
                         "64 = the L1 tiles' query chunk")
    ap.add_argument("--workload", default="gauss", choices=["gauss", "words", "dna", "zipf2d", "wordvec", "multicol",
                                                         "serving"],
                    help="gauss (the headline line); the others time the remaining configurations alone")
    ap.add_argument("--no-others", action="store_true", help="headline only: skip the other workloads")
    ap.add_argument("--other-steps", type=int, default=5, help="timed steps of the other workloads")
    ap.add_argument("--other-cpu-seconds", type=float, default=8.0)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "gauss":
        run_ours(args)
    else:
        run_config(args)


if __name__ == "__main__":
    main()
