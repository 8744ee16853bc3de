"""Benchmark: batched exact L2 kNN over a GTS index on GB300.

Workload (the headline configuration): 1,000,000 float32 vectors of dim 128
from a mixture of 64 isotropic Gaussians (centres uniform in [-1, 1], sigma
0.1, seed 0); 10,000 kNN queries, k = 10, from the same mixture (seed 1);
node capacity 20, h = 4 (Algorithm 1).  One step = one gts_knn call over the
whole 10,000-query batch: pivot distances, node pruning, the kNN threshold,
the list-table scan, verification and selection, all on the GPU.

Prints ONE JSON line (rank 0).  `value` is queries/s over all ranks with the
index and queries resident in HBM; `e2e` is the same metric through the C
ABI with pinned host queries and host results (copies inside the timed
region).  The index (X 512 MB, table 16 MB) is larger than L2 (129 MB), so no
explicit flush runs between steps.

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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per launch of the dominant kernel from one ncu capture (profiles/):
# k_tile_l2_tc at half size, 0.459 GB read + write (node rows and the node x
# query leaf-mask matrix), both of which double at full size.  None once the
# kernel has changed since the counters were taken.
TRAFFIC = {"kernel": "tile", "bytes_per_launch": 0.92e9}


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


def peaks():
    try:
        with open(MEASURED) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def tensor_peak():
    """Sustained dense bf16 TFLOP/s (a kernel timed inside a long step)."""
    try:
        with open(MEASURED) as f:
            m = json.load(f)
        return float(m["bf16_tflops_sustained"]), "measured"
    except Exception:
        return 1700.0, "fallback"


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


def algorithmic_bytes(stage: str, st: dict, dim: int, h: int, C: int) -> float:
    """Bytes the algorithm must move for one launch-set of a stage (see the
    design notes for the per-unit figures)."""
    if stage == "tile":
        # per work item (a 128-row block of a last-level node): the rows as split
        # bf16 (hi + lo), their table entries, norms and delete marks; per
        # (query, node) entry: the query as split bf16, its path distances and
        # metadata; per kept pair: (query, row) out
        dim_p = (dim + 63) // 64 * 64
        return (st["tiles"] * 128 * (4 * dim_p + h * 4 + 4 + 8)
                + st["tile_entries"] * (4 * dim_p + h * 4 + 8 + 4 + 4 + 8 + 4) + C * 8)
    if stage == "verify":
        return C * (dim * 4 + 4 + 4 + 4)            # candidate row + (query, row) + distance out
    if stage == "leaf_scan":
        return st["scanned_rows"] * (h * 4 + 8) * 2 + C * 8   # count and write passes, + candidates out
    if stage == "select":
        return C * (4 + 4 + 8) + st["rechecks"] * dim * 4
    if stage == "pivot_dist":
        return st["pivot_dist"] * (dim * 4 + 12)
    if stage == "expand":
        return st["frontier"] * (4 * 4 + 20 * 12)
    return 0.0


def max_over_ranks(x: float, dist, device: str) -> float:
    """The largest of the ranks' values (the slowest rank's time)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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

    def step_prec(p, timing=False):
        r = ix.knn(Qd, Kd, precision=p, result_on_device=True, timing=timing)
        st = r.stats
        r.free()
        return st

    def step(timing=False):
        return step_prec(prec, timing)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # ---- timed region: device-resident inputs
    stage_ms, stage_launch = {}, {}
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
            st = step(timing=True)
            marks[i + 1].record(stream)
            stats0 = stats0 or st
            launches += st["launches"]
            for kk, v in st["stage_ms"].items():
                stage_ms[kk] = stage_ms.get(kk, 0.0) + v
            for kk, v in st["stage_launches"].items():
                stage_launch[kk] = stage_launch.get(kk, 0) + v
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
    # ---- roofline of the dominant kernel (stage)
    dom = max(stage_ms, key=lambda s: stage_ms[s])
    C = stats0["candidates"]
    dom_ms_per_step = stage_ms[dom] / args.steps
    launches_dom = stage_launch[dom] / args.steps
    hbm, src = peaks()
    if dom == "tile" and prec == "bf16":
        # a contraction on the tensor cores: 2 D flops for every (query, row)
        # pair the tiles verify, against the sustained bf16 peak (the kernel
        # runs inside a long step); the split-bf16 form executes 3 products
        flops = stats0["tile_pairs"] * 2 * dim
        tf, tsrc = tensor_peak()
        sec = dom_ms_per_step / 1e3
        achieved = flops / sec / 1e12 if dom_ms_per_step > 0 else 0.0
        roof = {"bound": "tensor", "kernel": dom, "achieved": round(achieved, 1), "peak": tf, "unit": "TFLOP/s",
                "frac": round(achieved / tf, 4), "peak_source": tsrc,
                "traffic": TRAFFIC["bytes_per_launch"] if TRAFFIC["kernel"] == dom else None,
                "launches_per_step": launches_dom, "ms_per_step": round(dom_ms_per_step, 4),
                "executed_tflops": round(3 * achieved, 1),
                "hbm_algorithmic_gbs": round(algorithmic_bytes(dom, stats0, dim, info["h"], C) / sec / 1e9, 1)}
    else:
        alg = algorithmic_bytes(dom, stats0, dim, info["h"], C)
        achieved = alg / (dom_ms_per_step / 1e3) / 1e9 if dom_ms_per_step > 0 else 0.0
        roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_source": src,
                "traffic": TRAFFIC["bytes_per_launch"] if TRAFFIC["kernel"] == dom else None,
                "launches_per_step": launches_dom, "ms_per_step": round(dom_ms_per_step, 4)}
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
        "stage_ms_per_step": {kk: round(v / args.steps, 4) for kk, v in stage_ms.items()},
        "counters_per_step": {kk: v for kk, v in stats0.items() if not isinstance(v, dict)},
        "clocks": clocks.summary(),
    }
    if prec == "bf16" and not args.no_fp32_compare:
        # the plain FP32 single-batch path on the same index and queries
        for _ in range(1):
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
    if rank == 0 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(X, Q, k, budget_s=args.cpu_seconds)
    ix.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the other workloads (parity-test configurations; not the headline line)

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


def run_config(args):
    """Time one of the other workloads: words (edit range, r = 2), dna (edit
    range, r = 8), zipf2d (10M 2-D points, L2 range at ~0.01% selectivity,
    interleaved with stream updates and one batch update)."""
    import torch
    import paper_2404_00966_gb300 as gts
    from paper_2404_00966_gb300 import build_ext
    import synth

    build_ext.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    wl_name = args.workload
    prec = args.precision
    extra = {}
    if wl_name in ("words", "dna"):
        if wl_name == "words":
            wl = synth.words_like()
        else:   # --scale < 1: fewer seeds and queries (profiling only)
            wl = synth.dna_like() if args.scale >= 1.0 else synth.dna_like(
                n_seeds=max(100, int(10_000 * args.scale)), nq=max(100, int(20_000 * args.scale)))
        objs = _dev_strings(wl.objects)
        queries = _dev_strings(wl.queries)
        radii = torch.from_numpy(wl.radii).cuda()
        t0 = time.perf_counter()
        ix = gts.Index.build(objs, "edit", n_pivots=wl.n_pivots, fanout=wl.fanout, root_pivot=0)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        nq = wl.nq

        def step(timing=False):
            r = ix.range(queries, radii, precision=prec, result_on_device=True, timing=timing)
            st = r.stats
            r.free()
            return st
        metric = f"range queries/s at oracle-exact results (edit, r={int(wl.radii[0])})"
        host_q = wl.queries
    elif wl_name == "zipf2d":
        wl = synth.zipf_clusters_2d(nq=100_000)
        Xd = torch.from_numpy(wl.objects).cuda()
        t0 = time.perf_counter()
        ix = gts.Index.build(Xd, "l2", fanout=20, root_pivot=0, cache_limit=4096)
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        # one global radius with a mean result count of ~1,000 (0.01%) over 1,000
        # calibration queries: bisection on the range-query counts
        cal = torch.from_numpy(wl.queries[:1000]).cuda()
        r = calibrate_radius(ix, cal, 1000.0, torch)
        extra["radius"] = r
        nq = 10_000
        Qall = torch.from_numpy(wl.queries).cuda()
        radii = torch.full((nq,), r, dtype=torch.float32, device="cuda")
        upd = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 10_000, seed=2)
        bulk = synth.zipf_points(wl.extra["centers"], wl.extra["weights"], 0.01, 500_000, seed=5)
        drng = np.random.default_rng(3)
        state = {"round": 0, "next_ins": 0, "update_s": 0.0}

        def step(timing=False):
            i = state["round"] % 10
            qb = Qall[i * nq:(i + 1) * nq]
            res = ix.range(qb, radii, precision=prec, result_on_device=True, timing=timing)
            st = res.stats
            res.free()
            # 10% updates between query batches: 500 inserts + 500 deletes
            u0 = time.perf_counter()
            a = state["next_ins"] % 9_500
            ix.insert(upd[a:a + 500])
            state["next_ins"] += 500
            info = ix.info()
            ix.delete(drng.integers(0, info["next_id"], size=500))
            if state["round"] == 5:
                ix.batch_update(bulk)   # one batch update: rebuild with 500,000 more points
            torch.cuda.synchronize()
            state["update_s"] += time.perf_counter() - u0
            state["round"] += 1
            return st
        metric = "range queries/s at oracle-exact results (L2, ~0.01% selectivity, 10% stream updates)"
        host_q = None
    else:
        raise SystemExit(f"unknown workload {wl_name}")
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stage_ms, launches, stats0 = {}, 0, None
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clocks:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if wl_name == "zipf2d":
            state["update_s"] = 0.0
        e0.record(stream)
        for _ in range(args.steps):
            st = step(timing=True)
            stats0 = stats0 or st
            launches += st["launches"]
            for kk, v in st["stage_ms"].items():
                stage_ms[kk] = stage_ms.get(kk, 0.0) + v
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if wl_name == "zipf2d":
        # queries/s over the query work only: the update calls are timed apart
        qms = ms - 1e3 * state["update_s"]
        extra["update_ms_per_round"] = round(1e3 * state["update_s"] / args.steps, 3)
    else:
        qms = ms
    value = nq * args.steps / (qms / 1e3)
    out = {"metric": metric, "value": round(value, 1), "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(qms / args.steps, 4), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "int32" if wl_name in ("words", "dna") else ("bf16+f64" if prec == "bf16" else "f32+f64"),
           "data": "synthetic",
           "config": {"workload": wl_name, "n": ix.info()["n_tree"], "nq": nq, "build_s": round(build_s, 3),
                      "precision": prec, **extra},
           "gpu_launches": int(launches),
           "stage_ms_per_step": {kk: round(v / args.steps, 4) for kk, v in stage_ms.items()},
           "counters_per_step": {kk: v for kk, v in stats0.items() if not isinstance(v, dict)},
           "clocks": clocks.summary()}
    if host_q is not None:
        # edit distance: DP cells (full-matrix equivalent) of the pivot and
        # verification stages per second
        lq = float(np.mean(np.diff(host_q.offsets)))
        lo = float(np.mean(np.diff(wl.objects.offsets)))
        rates = {}
        for stage, pairs in (("pivot_dist", stats0["pivot_dist"]), ("verify", stats0["candidates"])):
            sec = stage_ms.get(stage, 0.0) / args.steps / 1e3
            if sec > 0:
                rates[stage] = {"dp_cells_per_s": pairs * lq * lo / sec}
        if rates:
            dom = max(rates, key=lambda k: stage_ms[k])
            if wl_name == "dna" and dom == "pivot_dist":
                # the bit-parallel DP keeps the ALU pipe 85.3% busy (ncu, profiles/
                # pivdist_str_dna_200k_r8.md): the cell rate at a full pipe is the peak
                busy = 0.853
                out["roofline"] = {"bound": "alu", "kernel": dom, "unit": "Tcell/s",
                                   "achieved": round(rates[dom]["dp_cells_per_s"] / 1e12, 3),
                                   "peak": round(rates[dom]["dp_cells_per_s"] / busy / 1e12, 3),
                                   "peak_source": "ncu ALU-pipe utilisation of k_pivdist_str", "frac": busy,
                                   "dp_cells_per_s": {k: round(v["dp_cells_per_s"], 1) for k, v in rates.items()},
                                   "traffic": None}
            else:
                out["roofline"] = {"bound": "latency", "kernel": dom, "unit": "Tcell/s",
                                   "achieved": round(rates[dom]["dp_cells_per_s"] / 1e12, 3), "peak": None,
                                   "frac": None,
                                   "dp_cells_per_s": {k: round(v["dp_cells_per_s"], 1) for k, v in rates.items()},
                                   "traffic": None}
    if not args.no_cpu and host_q is not None:
        import oracle
        oracle.build()
        m = min(host_q.n, args.ref_sample)
        sub = host_q.take(np.arange(m))
        t0 = time.perf_counter()
        oracle.range_query("edit", wl.objects, sub, wl.radii[:m])
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": round(m / dt, 3), "unit": "queries/s", "cores": oracle.threads(),
                               "kind": "oracle", "sample": f"{m} queries, brute-force banded edit distance"}
    ix.close()
    print(json.dumps(out), flush=True)


def run_serving(args):
    """Open-loop serving: 2,000,000 x 256 uniform vectors, L1; requests arrive
    as a Poisson stream at 50,000/s (half range queries with a radius of ~100
    results, half kNN with k uniform in 1..100) and are served by the
    continuous-batching loop under a 16 GB admission budget.  Reports the
    served requests/s and the p50 / p99 latency from submit to result."""
    import torch
    import paper_2404_00966_gb300 as gts
    from paper_2404_00966_gb300 import build_ext
    import synth

    build_ext.build()
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    nreq = args.requests
    wl = synth.uniform_cube(n=2_000_000, dim=256, nq=nreq + 512)
    t0 = time.perf_counter()
    ix = gts.Index.build(torch.from_numpy(wl.objects).cuda(), "l1", fanout=20, root_pivot=0)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    cal = torch.from_numpy(wl.queries[nreq:nreq + 256]).cuda()
    radius = calibrate_radius(ix, cal, 100.0, torch, iters=16)
    is_knn, ks = synth.mixed_requests(nreq, seed=1)
    arrivals = synth.poisson_arrivals(nreq, args.rate, seed=1)
    sv = gts.Server(ix, max_batch=args.max_batch, n_streams=3, precision=args.precision, result_budget=16 << 30)
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
    value = nreq / span
    out = {"metric": "served mixed range/kNN requests/s (L1, Poisson arrivals, 16 GB admission budget); p50/p99 ms",
           "value": round(value, 1), "unit": "requests/s", "n_gpus": 1, "steps": 1, "warmup": 1,
           "ms_per_step": round(1e3 * span, 2), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": "uniform_2Mx256_l1_serving", "n": 2_000_000, "dim": 256, "requests": nreq,
                      "arrival_rate": args.rate, "radius": radius, "build_s": round(build_s, 3),
                      "max_batch": args.max_batch, "streams": 3, "precision": args.precision},
           "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3), "p99": round(float(np.percentile(lat, 99)), 3),
                          "mean": round(float(lat.mean()), 3), "max": round(float(lat.max()), 3)},
           "offered_span_s": round(float(arrivals[-1]), 4), "server": st, "clocks": clocks.summary()}
    ix.close()
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
    ap.add_argument("--workload", default="gauss", choices=["gauss", "words", "dna", "zipf2d", "serving"],
                    help="gauss (the headline line); the others time the remaining configurations")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "gauss":
        run_ours(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_config(args)


if __name__ == "__main__":
    main()
