#!/usr/bin/env python
"""Benchmark of the GraphZero counting hot path on GB300 (one JSON line on rank 0).

Default workload (k-clique counting with degree orientation): R-MAT scale 20,
edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), seed 20; one step =
plan K4 and K5 (host planner), orient the device-resident graph (GPU reindex +
out-list build), build the clique rows of the new view (gz_prepare), count K4
and K5 with one merged program (gz_count_merged: one fused pass over the root
pairs, exact uint64), counts back to the host. Metric: intersected elements per second, E / step time, where E is
the number of list elements the bounded linear scans of the paper's nested
loops consume (computed by the CPU oracle and stored in tests/golden).

Other workloads (--config): triangle (ER 4096, plain method), patterns (R-MAT
22, five patterns on the oracle's sampled root ranges, one per call and all in
one batched call), pattern_samples (one range per pattern, for profiling),
batched (64 queries over 16 graphs, one launch vs one per launch), served
(Poisson request stream on a device-resident R-MAT graph, scale 24 by default,
against FIFO one query per launch), motifs (merged vs separate programs),
schedules, planner.
The default run also prints short triangle / patterns / batched records
(--no-subconfigs skips them).

--impl reference times the CPU oracle on a bounded sample of the same workload.
Under torchrun each rank runs a replica of the workload on its own GPU (weak
scaling, no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "intersected elements/s (count time; E/t as % of HBM peak)"
UNIT = "elem/s"
GOLDEN = os.path.join(ROOT, "tests", "golden")
PROFILES = os.path.join(ROOT, "profiles")


# ------------------------------------------------------------------ distributed helpers

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def aggregate(dist, elapsed_s: float, units: float):
    """Max of elapsed over ranks and sum of units over ranks (whole-job totals)."""
    if dist is None:
        return elapsed_s, units
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ------------------------------------------------------------------ measurement helpers

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the source of k_clique_warp and the device helpers it runs (the
    kernel the roofline figures are for); the whole file if the markers move."""
    src = open(os.path.join(ROOT, "paper_1911_12877_gb300", "csrc", "gz_clique.cu")).read()
    parts = []
    for a, b in (("// Row stride (32-bit words) of the bitset rows", "// Index of x in sorted O[0, n)"),
                 ("// K = 4 and K = 5 on roots with 32 < |O| <= max_out: k_clique_warp.",
                  "// Roots whose out-list is too long for shared-memory rows")):
        i, j = src.find(a), src.find(b)
        if i < 0 or j < i:
            parts = [src]
            break
        parts.append(src[i:j])
    h = hashlib.sha256()
    for p in parts:
        h.update(p.encode())
    return h.hexdigest()[:16]


PROFILE_K5 = "k_clique_warp_k5_rmat20.json"


def profiled(name: str):
    """Figures of a committed ncu summary (DRAM bytes per launch, pipe use), if
    it was taken on the current kernel source; else None."""
    path = os.path.join(PROFILES, name)
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("kernel_source_sha") != kernel_source_hash():
        return None
    return d


#: popcount results per clock per SM: the instruction runs on the SM's XU pipe,
#: a quarter of the 64-lane integer ALU rate (NVIDIA's arithmetic-instruction
#: throughput table for compute capabilities 7.x-10.x); the committed ncu
#: summary of the clique kernel states the XU pipe's own utilisation beside it
XU_POPC_PER_CLK_SM = 16


def clique_roofline(words, kernel_s, e_elems, clocks, sms, prof):
    """Roofline of the fused K4 + K5 clique count (one gz_count_merged call). Its
    work is bitset word operations (one 32-bit word of a candidate set ANDed
    and popcounted or walked), counted exactly by the oracle's bitset work
    measure for the K4 and the K5 loops; every word of a last loop takes one
    popcount, so the bound is the SMs' popcount rate at the sampled SM clock."""
    mhz = clocks.get("sm_mhz") or 2070.0
    peak = XU_POPC_PER_CLK_SM * sms * mhz * 1e6 / 1e9
    achieved = words / kernel_s / 1e9
    hbm, hbm_kind = measured_peaks()
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    return {"bound": "alu", "kernel": "k_clique_small<5> + k_clique_warp<5, fused K4> (K4 + K5 counts)",
            "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Gword-op/s",
            "frac": round(achieved / peak, 4), "traffic": traffic,
            "peak_kind": f"derived: {XU_POPC_PER_CLK_SM} popcounts/clk/SM x {sms} SMs x {mhz:.0f} MHz "
                         "(median SM clock sampled during the timed region)",
            "kernel_ms": round(kernel_s * 1e3, 3), "algorithmic_words": words,
            "e_rate_over_hbm_peak": round(4.0 * e_elems / kernel_s / 1e9 / hbm, 3),
            "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind,
            "dram_frac": (round(traffic / kernel_s / 1e9 / hbm, 6) if traffic else None),
            "xu_pipe_pct_ncu": prof.get("xu_pipe_pct") if prof else None,
            "issue_active_pct_ncu": prof.get("issue_active_pct") if prof else None,
            "note": "achieved = bitset word operations of the K4 and K5 loops (oracle, exact) / time of "
                    "the fused count (CUDA events); e_rate_over_hbm_peak = 4 x E / t over the HBM copy peak, E = list "
                    "elements the paper's bounded linear scans would consume: the bitset kernel reads each "
                    "root's rows from shared memory, so that ratio exceeds 1 and is not a roofline fraction"}


def flush_l2(buf):
    buf.add_(1)  # writes a buffer larger than L2 (129 MB)


# ------------------------------------------------------------------ workloads

def load_golden(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        raise SystemExit(f"missing {path}: run tests/golden/make_golden.py")
    return json.load(open(path))


def clique_workload():
    import synthetic as S
    g = S.rmat_clique()
    gold = load_golden("clique_rmat20.json")
    if gold["nnz"] != g.nnz:
        raise SystemExit("golden clique_rmat20.json does not match the generated graph")
    return g, gold


def cpu_baseline_clique(g, gold, target_s: float = 12.0, max_s: float = 40.0, nthreads: int = 0):
    """The oracle as it stands on a bounded sample: roots in 16 evenly spaced
    ranges of width w of the reindexed graph, K4 and K5, all host threads (or
    nthreads)."""
    import oracle as O
    from synthetic.patterns import adjacency
    go, _ = O.reindex(g)
    pats = [(adjacency("k4"), gold["k4"]["order"]), (adjacency("k5"), gold["k5"]["order"])]
    starts = [i * (g.n // 16) + 4096 for i in range(16)]  # skip the very top hubs
    w, t, e = 1, 0.0, 0
    while True:
        t0 = time.perf_counter()
        e = 0
        for a, order in pats:
            for s in starts:
                e += O.count_nested(a, order, go, s, min(g.n, s + w), nthreads=nthreads)[1]
        t = time.perf_counter() - t0
        if t >= target_s or t * 2 > max_s or w >= g.n // 16:
            break
        w = max(w * 2, int(w * target_s / max(t, 1e-3) * 0.9))
    cores = nthreads if nthreads > 0 else O.threads()
    return {"value": e / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"K4+K5 on R-MAT 20 (reindexed), roots in 16 ranges of {w} ids "
                      f"starting at i*n/16+4096; E={e} in {t:.2f} s on {cores} thread(s)"}, w, starts


def run_clique(args, dist, world, rank, local):
    import torch
    import paper_1911_12877_gb300 as gz
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    g, gold = clique_workload()
    e_k4, e_k5 = gold["k4"]["elems"], gold["k5"]["elems"]
    e_total = e_k4 + e_k5
    G = gz.Graph.from_csr(g)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2

    count_ev = []

    def step(record=False):
        p4, p5 = gz.Plan("k4"), gz.Plan("k5")  # planner (host)
        G.orient()
        gz.prepare(p5, G, orientation=True)  # the reoriented view's clique rows
        if record:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
        # one merged program for both patterns: the K4 loops are a prefix of the
        # K5 loops, so one pass over the root pairs yields both counts (timed
        # apart for the roofline: the clique kernels only)
        c4, c5 = gz.count_merged([p4, p5], G, orientation=True)
        if record:
            b.record(stream)
            count_ev.append((a, b))
        return c4, c5

    for _ in range(args.warmup):
        counts = step()
    if counts[0] != gold["k4"]["count"]:
        raise SystemExit(f"K4 count {counts[0]} != oracle {gold['k4']['count']}")
    if "count" in gold["k5"] and counts[1] != gold["k5"]["count"]:
        raise SystemExit(f"K5 count {counts[1]} != oracle {gold['k5']['count']}")
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = gz.kernel_launches()
    evs = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            counts = step(record=True)
            b.record(stream)
            evs.append((a, b))
            if i + 1 < args.steps:
                flush_l2(flush)
        torch.cuda.synchronize()
    launches = gz.kernel_launches() - launches0
    barrier(dist)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    count_ms = [a.elapsed_time(b) for a, b in count_ev]
    elapsed = sum(step_ms) / 1e3
    elapsed_max, units = aggregate(dist, elapsed, e_total * args.steps)
    value = units / elapsed_max
    count_s = statistics.mean(count_ms) / 1e3
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    roofline = clique_roofline(gold["k4"]["bitset_words"] + gold["k5"]["bitset_words"], count_s, e_total, clocks,
                               sms, profiled(PROFILE_K5))

    # end to end through the C ABI with host buffers (pinned), copies inside the timing
    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(g.row_ptr).pin_memory()
        col_h = torch.from_numpy(g.col).pin_memory()
        import ctypes
        e2e_t = []
        for i in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = ctypes.c_void_p()
            gz._check(gz.lib().gz_load_csr(rp_h.data_ptr(), col_h.data_ptr(), g.n, g.nnz, 0, 0,
                                           stream.cuda_stream, ctypes.byref(h)), "gz_load_csr")
            Gh = gz.Graph.__new__(gz.Graph)
            Gh.handle, Gh.n, Gh.nnz, Gh._keep = h, g.n, g.nnz, None
            Gh.orient()
            p4, p5 = gz.Plan("k4"), gz.Plan("k5")
            gz.prepare(p5, Gh, orientation=True)
            c = tuple(gz.count_merged([p4, p5], Gh, orientation=True))
            Gh.close()
            torch.cuda.synchronize()
            e2e_t.append(time.perf_counter() - t0)
            if c != counts:
                raise SystemExit("end-to-end counts differ from the device-resident run")
        t_e2e, u_e2e = aggregate(dist, sum(e2e_t), e_total * len(e2e_t))
        e2e = {"value": u_e2e / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * (g.n + 1) + 4 * g.nnz,
               "d2h_bytes_per_step": 16, "ms_per_step": round(1e3 * t_e2e / len(e2e_t), 3)}

    # the two host/HBM steps of the path on their own: the planner (Sec. 7.3 quotes
    # 0.6 ms for the size-7 chordal cycle) and the orientation pass (Table 3)
    plan_ms = {}
    for name in ("k5", "house", "chordal7"):
        ts = []
        for _ in range(20):
            t0 = time.perf_counter()
            gz.Plan(name)
            ts.append(1e3 * (time.perf_counter() - t0))
        plan_ms[name] = round(statistics.median(ts), 4)
    o_ms = []
    for _ in range(5):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.orient()
        b.record(stream)
        torch.cuda.synchronize()
        o_ms.append(a.elapsed_time(b))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_clique(g, gold)[0]
        cpu["single_thread"] = cpu_baseline_clique(g, gold, target_s=8.0, max_s=25.0, nthreads=1)[0]
    subs = None
    if rank == 0 and world == 1 and not args.no_subconfigs:
        subs = sub_records(args, dist, world, rank, local)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * elapsed_max / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": "k-clique K4+K5 with degree orientation, R-MAT scale 20 ef 16 "
                               "seed 20 (a,b,c,d)=(.57,.19,.19,.05)", "n": g.n, "nnz": g.nnz,
                   "parallelism": f"replicas{world}", "l2": "flushed between timed steps",
                   "step": "plan K4,K5 + GPU orient + clique rows (gz_prepare) + count K4 and K5 (one merged program, gz_count_merged)"},
        "counts": {"k4": counts[0], "k5": counts[1]},
        "elems_per_step": e_total,
        "step_ms": [round(x, 3) for x in step_ms],
        "plan_ms": plan_ms, "orient_ms": round(statistics.median(o_ms), 3),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clocks,
    }
    if subs is not None:
        line["subconfigs"] = subs
    return line


def sub_records(args, dist, world, rank, local):
    """Short runs of the triangle (ER 4096), arbitrary-pattern (R-MAT 22 oracle
    samples, counts re-checked) and batched (64 queries, counts checked against
    the oracle's values) workloads, each with its own clock record."""
    import argparse as _ap
    out = {}
    for name, fn, kw in (("triangle", run_triangle, {"steps": 20}),
                         ("patterns_rmat22", run_patterns, {"steps": 3}),
                         ("batched", run_batched, {"steps": 2, "tune_min_ms": 1e12})):
        a = _ap.Namespace(**vars(args))
        for k, v in kw.items():
            setattr(a, k, v)
        a.warmup = 1
        t0 = time.perf_counter()
        with ClockSampler(local) as clk:
            rec = fn(a, dist, world, rank, local)
        rec["clocks"] = clk.summary()
        rec["wall_s"] = round(time.perf_counter() - t0, 2)
        for k in ("n_gpus", "steps", "warmup", "scaling", "vs_baseline", "dtype", "data"):
            rec.pop(k, None)
        out[name] = rec
    return out


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, as it stands, on a bounded sample per step."""
    if rank != 0:
        return None
    import oracle as O
    from synthetic.patterns import adjacency
    g, gold = clique_workload()
    base, w, starts = cpu_baseline_clique(g, gold, target_s=6.0, max_s=20.0)
    go, _ = O.reindex(g)
    pats = [(adjacency("k4"), gold["k4"]["order"]), (adjacency("k5"), gold["k5"]["order"])]

    def step():
        e = 0
        for a, order in pats:
            for s in starts:
                e += O.count_nested(a, order, go, s, min(g.n, s + w))[1]
        return e

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    e = 0
    for _ in range(args.steps):
        e += step()
    t = time.perf_counter() - t0
    v = e / t
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "k-clique K4+K5 with degree orientation, R-MAT scale 20 ef 16 "
                                   "seed 20 (bounded root sample per step)", "n": g.n, "nnz": g.nnz},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": O.threads(),
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ other workloads


def _time_counts(fn, reps, stream, flush=None):
    """CUDA-event time of fn() per call (ms list), after one untimed call."""
    import torch
    out = fn()
    ms = []
    for _ in range(reps):
        if flush is not None:
            flush_l2(flush)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        if r != out:
            raise SystemExit(f"count changed between repetitions: {out} vs {r}")
    return out, ms


def _summary(ms):
    s = sorted(ms)
    return {"median_ms": round(statistics.median(s), 4), "min_ms": round(s[0], 4),
            "p90_ms": round(s[min(len(s) - 1, int(0.9 * len(s)))], 4)}


def _line(metric, value, unit, args, world, ms_per_step, config, hib=True, **kw):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": hib,
         "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
         "config": config}
    d.update(kw)
    return d


def run_triangle(args, dist, world, rank, local):
    """Triangle counting, plain method (restrictions on the original ids, no reindex):
    ER G(4096, 16/4095), seed 1. L2-resident and launch-latency bound."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    g = S.er_triangle()
    gold = load_golden("er_triangle.json")
    G = gz.Graph.from_csr(g)
    p = gz.Plan("triangle")
    reps = max(20, args.steps)
    l0 = gz.kernel_launches()
    c, ms = _time_counts(lambda: gz.count(p, G, orientation=False), reps, stream)
    launches = gz.kernel_launches() - l0
    if c != gold["triangle"]["count"]:
        raise SystemExit(f"triangle count {c} != oracle {gold['triangle']['count']}")
    e = gold["triangle"]["elems"]
    med = statistics.median(ms)
    return _line("intersected elements/s (count time)", e / (med / 1e3), UNIT, args, world, med,
                 {"workload": "triangle, plain method (original ids), ER n=4096 p=16/4095 seed 1",
                  "n": g.n, "nnz": g.nnz, "l2": "resident (270 KB CSR); not flushed"},
                 count=c, elems=e, count_us=round(med * 1e3, 2), timing=_summary(ms),
                 gpu_launches=launches, note="launch-latency bound: % of HBM is not meaningful")


def run_patterns(args, dist, world, rank, local):
    """Arbitrary patterns with restrictions and generalized orientation on R-MAT
    (default scale 22, ef 16, seed 22): c4, diamond, paw, house, chordal5.

    Per pattern: the oracle's sampled root ranges (hub blocks to low-degree
    blocks) are counted and timed, each count checked against the stored oracle
    value, and E over those ranges / their count time gives the throughput (one
    range per call). batched_ranges times the same ranges of all patterns in one
    gz_count_batch_ranges call. The full count is timed for the patterns in
    --full (its cost on this graph is listed in the design notes for the
    others)."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    from synthetic.patterns import PATTERN_SET
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    scale = args.scale or 22
    g = S.rmat(scale, 16, scale)
    gold = None
    if scale == 22 and os.path.exists(os.path.join(GOLDEN, "patterns_rmat22.json")):
        gold = load_golden("patterns_rmat22.json")
    G = gz.Graph.from_csr(g)
    _, t_or = _time_counts(lambda: (G.orient(), 0)[1], 3, stream)
    names = args.patterns.split(",") if args.patterns else PATTERN_SET
    if args.full:
        full = set(args.full.split(","))
    else:  # on R-MAT 22 one full count takes 38 s (diamond) to hours (house)
        full = set() if scale == 22 else set(names)
    peak = measured_peaks()[0]
    res = {}
    tot_e, tot_ms = 0, 0.0
    l0 = gz.kernel_launches()
    for name in names:
        p = gz.Plan(name)
        r = {}
        if gold and name in gold["patterns"]:
            e_s, ms_s = 0, 0.0
            for lo, hi, want, e in gold["patterns"][name]["samples"]:
                got, ms = _time_counts(lambda: gz.count(p, G, True, lo, hi), args.steps, stream)
                if got != want:
                    raise SystemExit(f"{name} roots [{lo},{hi}): {got} != oracle {want}")
                e_s += e
                ms_s += statistics.median(ms)
            r["sampled"] = {"ranges": len(gold["patterns"][name]["samples"]), "elems": e_s,
                            "ms": round(ms_s, 3), "elems_per_s": e_s / (ms_s / 1e3),
                            "hbm_frac_algorithmic": round(4 * e_s / (ms_s / 1e3) / 1e9 / peak, 4),
                            "oracle_parity": "ok"}
            tot_e += e_s
            tot_ms += ms_s
        if name in full:
            c, ms = _time_counts(lambda: gz.count(p, G, orientation=True), args.steps, stream)
            r["full"] = {"count": c, **_summary(ms)}
        res[name] = r
    launches = gz.kernel_launches() - l0
    value = tot_e / (tot_ms / 1e3) if tot_ms > 0 else None
    extra = {}
    if gold:
        # the same sampled ranges, all patterns at once: one gz_count_batch_ranges
        # call (a few roots per range leave most of the device idle when each
        # range is counted alone)
        plans, ranges, wants, e_b = [], [], [], 0
        for name in names:
            if name not in gold["patterns"]:
                continue
            p = gz.Plan(name)
            for lo, hi, want, e in gold["patterns"][name]["samples"]:
                plans.append(p)
                ranges.append((lo, hi))
                wants.append(want)
                e_b += e
        nb = len(plans)
        l1 = gz.kernel_launches()
        got, ms = _time_counts(lambda: gz.count_batch_ranges(plans, [G] * nb, [True] * nb, ranges),
                               args.steps, stream)
        if got != wants:
            bad = [(ranges[i], got[i], wants[i]) for i in range(nb) if got[i] != wants[i]]
            raise SystemExit(f"batched ranges differ from the oracle: {bad[:3]}")
        med = statistics.median(ms)
        extra["batched_ranges"] = {
            "queries": nb, "elems": e_b, **_summary(ms), "elems_per_s": e_b / (med / 1e3),
            "hbm_frac_algorithmic": round(4 * e_b / (med / 1e3) / 1e9 / peak, 4),
            "speedup_vs_one_range_per_call": round(tot_ms / med, 3) if med > 0 else None,
            "gpu_launches_per_call": (gz.kernel_launches() - l1) // (args.steps + 1),
            "oracle_parity": "ok"}
    return _line("intersected elements/s over the oracle's sampled root ranges", value, UNIT, args,
                 world, tot_ms,
                 {"workload": f"c4, diamond, paw, house, chordal5 with restrictions + orientation, "
                              f"R-MAT scale {scale} ef 16 seed {scale}", "n": g.n, "nnz": g.nnz,
                  "l2": "graph larger than L2; not flushed between ranges"},
                 patterns=res, orient_ms=_summary(t_or), gpu_launches=launches, **extra)


def run_pattern_samples(args, dist, world, rank, local):
    """One count per pattern on the oracle's heaviest sampled root range of R-MAT
    scale 22 (the range with the most list elements E), each checked against the
    oracle's value: a short fixed launch sequence for profiling the general
    kernel (one k_enumerate_one launch per pattern, plus its split pass)."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    from synthetic.patterns import PATTERN_SET
    torch.cuda.set_device(local)
    g = S.rmat(22, 16, 22)
    gold = load_golden("patterns_rmat22.json")
    G = gz.Graph.from_csr(g).orient()
    names = args.patterns.split(",") if args.patterns else PATTERN_SET
    out = {}
    t0 = time.perf_counter()
    for name in names:
        lo, hi, want, e = max(gold["patterns"][name]["samples"], key=lambda x: x[3])
        got = gz.count(gz.Plan(name), G, True, lo, hi)
        if got != want:
            raise SystemExit(f"{name} roots [{lo},{hi}): {got} != oracle {want}")
        out[name] = {"roots": [lo, hi], "count": got, "elems": e}
    ms = 1e3 * (time.perf_counter() - t0)
    return _line("one count per pattern on its heaviest oracle sample", ms, "ms", args, world, ms,
                 {"workload": f"{names} on R-MAT scale 22 ef 16 seed 22 (oriented)"}, hib=False,
                 samples=out, oracle_parity="ok")


def run_batched(args, dist, world, rank, local):
    """64 queries (12 patterns) over 16 R-MAT graphs of scales 10..21 in one
    gz_count_batch call, before and after gz_autotune tuned the queries that take
    at least --tune-min-ms alone, against the same 64 run one per gz_count call.
    Every count is checked against the oracle's stored values."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    from synthetic.patterns import batch_queries
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    top = args.scale or 21
    idx = [i for i in range(16) if S.BATCH_SCALES[i] <= top]
    graphs = {i: gz.Graph.from_csr(S.batch_graph(i)).orient() for i in idx}
    table = [(gi, name) for gi, name in batch_queries() if gi in graphs]
    plans = {name: gz.Plan(name) for _, name in table}
    qp = [plans[n] for _, n in table]
    qg = [graphs[gi] for gi, _ in table]
    qo = [True] * len(table)
    l0 = gz.kernel_launches()
    untuned, ms_u = _time_counts(lambda: gz.count_batch(qp, qg, qo), args.steps, stream)
    lb = gz.kernel_launches() - l0
    plain, ms_p = _time_counts(lambda: [gz.count(p, G, True) for p, G in zip(qp, qg)], args.steps,
                               stream)
    if untuned != plain:
        raise SystemExit("batched counts differ from one-per-launch counts")
    # time each distinct query alone, then tune those that take long enough
    alone_ms = {}
    for (gi, name), p, G in zip(table, qp, qg):
        if (gi, name) not in alone_ms:
            alone_ms[(gi, name)] = statistics.median(_time_counts(lambda: gz.count(p, G, True), 1, stream)[1])
    t0 = time.perf_counter()
    tuned_sets = {}
    for (gi, name), ms in alone_ms.items():
        if ms >= args.tune_min_ms:
            tuned_sets[f"{gi}:{name}"] = gz.autotune(plans[name], graphs[gi], True)
    tune_s = time.perf_counter() - t0
    batch, ms_b = _time_counts(lambda: gz.count_batch(qp, qg, qo), args.steps, stream)
    if batch != plain:
        raise SystemExit("tuned batched counts differ from one-per-launch counts")
    parity = batched_oracle_parity(table, batch, plans, graphs)
    mb, mu, mp = statistics.median(ms_b), statistics.median(ms_u), statistics.median(ms_p)
    return _line("queries/s, batched (one gz_count_batch call, autotuned)", len(table) / (mb / 1e3),
                 "queries/s", args, world, mb,
                 {"workload": f"{len(table)} queries over {len(graphs)} R-MAT graphs (scales 10..{top}, "
                              f"ef 8..32, seeds 100+i), query table seed 4", "queries": len(table)},
                 untuned_queries_per_s=len(table) / (mu / 1e3), plain_queries_per_s=len(table) / (mp / 1e3),
                 speedup_vs_plain=mp / mb, speedup_tuned_vs_untuned=mu / mb, oracle_parity=parity,
                 batched=_summary(ms_b), untuned=_summary(ms_u), plain=_summary(ms_p),
                 tuned_queries=tuned_sets, tune_s=round(tune_s, 2),
                 gpu_launches_per_batch=lb // (args.steps + 1), counts=[int(x) for x in batch])


def batched_oracle_parity(table, counts, plans, graphs):
    """Checks the batched counts against the oracle's stored values: the full
    count where the oracle finished, else its sampled root ranges (counted here
    through gz_count_ex). Returns "ok" or exits."""
    import paper_1911_12877_gb300 as gz
    gold = load_golden("batched_table.json")
    full = sampled = 0
    for (gi, name), c in zip(table, counts):
        r = gold["results"].get(f"{gi}:{name}")
        if r is None:
            raise SystemExit(f"batched_table.json has no oracle value for graph {gi} {name}")
        if "count" in r:
            if c != r["count"]:
                raise SystemExit(f"batched graph {gi} {name}: {c} != oracle {r['count']}")
            full += 1
        else:
            for lo, hi, want, _ in r["samples"]:
                got = gz.count(plans[name], graphs[gi], True, lo, hi)
                if got != want:
                    raise SystemExit(f"batched graph {gi} {name} roots [{lo},{hi}): {got} != oracle {want}")
            sampled += 1
    return {"status": "ok", "full_counts": full, "sampled_ranges": sampled}


def _alone_time(gz, p, G, n, cap_s, piece_s=0.5):
    """Service time of one request alone, bounded: the roots are counted in
    consecutive ranges sized to take about piece_s each (from the previous
    range's rate, within 4x), hub end first, until all are counted or cap_s has
    passed. Returns (seconds, roots counted, count over them)."""
    import time as _t
    lo, width, total, spent = 0, 1, 0, 0.0
    while lo < n and spent < cap_s:
        hi = min(n, lo + width)
        t0 = _t.perf_counter()
        total += gz.count(p, G, True, lo, hi)
        dt = _t.perf_counter() - t0
        spent += dt
        lo = hi
        width = int(min(4 * width, max(width / 4, width * piece_s / max(dt, 1e-4)))) or 1
    return spent, lo, total


def run_served(args, dist, world, rank, local):
    """Poisson request stream over a device-resident R-MAT graph and its oriented
    copy: continuous batching (fast requests batched on free streams; a slow one
    at a time on a share of the device, so fast ones run beside it) against
    FIFO, one whole-graph query per launch in arrival order. The slow threshold
    is twice the median service time alone of the stream's patterns unless
    --heavy-ms is given.

    Default graph: R-MAT scale 24 (ef 16, seed 24). Each pattern of the request
    mix is first measured alone, bounded by --alone-cap seconds (roots counted in
    growing ranges, hub end first): a pattern whose count finishes within the cap
    joins the stream; the others (c4, diamond and the chordal 5-cycle need
    minutes per count on this graph) are reported with the roots they covered
    and the time, a lower bound of their service time. Every served and FIFO
    result must equal its count alone, and the oracle's sampled root ranges of
    the graph (tests/golden/served_rmat24.json) are counted and compared."""
    import numpy as np
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    from synthetic.patterns import SERVED_PATTERNS
    torch.cuda.set_device(local)
    scale = args.scale or 24
    g = S.rmat(scale, 16, scale)
    G = gz.Graph.from_csr(g).orient()
    names = args.patterns.split(",") if args.patterns else SERVED_PATTERNS
    alone, stream = {}, []
    for name in names:
        p = gz.Plan(name)
        secs, roots, cnt = _alone_time(gz, p, G, g.n, args.alone_cap)
        rec = {"roots_counted": roots, "of": g.n, "seconds": round(secs, 3)}
        if roots == g.n:
            import time as _t
            t0 = _t.perf_counter()
            c = gz.count(p, G, True)
            rec.update(count=c, whole_count_s=round(_t.perf_counter() - t0, 3))
            if c != cnt:
                raise SystemExit(f"{name}: whole count {c} != sum of its root ranges {cnt}")
            stream.append(name)
        else:
            rec["note"] = "cap reached: the full count takes longer than these seconds"
        alone[name] = rec
    parity = None
    if scale == 24 and os.path.exists(os.path.join(GOLDEN, "served_rmat24.json")):
        gold = load_golden("served_rmat24.json")
        if gold["nnz"] != g.nnz:
            raise SystemExit("served_rmat24.json does not match the generated graph")
        checked = 0
        for name, rec in gold["patterns"].items():
            p = gz.Plan(name)
            for lo, hi, want, _ in rec["samples"]:
                got = gz.count(p, G, True, lo, hi)
                if got != want:
                    raise SystemExit(f"served graph {name} roots [{lo},{hi}): {got} != oracle {want}")
                checked += 1
        parity = {"status": "ok", "sampled_ranges": checked}
    if not stream:
        raise SystemExit("no pattern of the mix finishes within --alone-cap")
    plans = [gz.Plan(n) for n in stream]
    counts_alone = [alone[n]["count"] for n in stream]
    mean_s = float(np.mean([alone[n]["whole_count_s"] for n in stream]))
    heavy_ms = args.heavy_ms or max(1.0, 2e3 * float(np.median([alone[n]["whole_count_s"] for n in stream])))
    nreq = args.requests or (300 if mean_s < 0.05 else max(6, int(60.0 / max(mean_s, 1e-3))))
    rates = args.rates or ("12.5,25,50,100,200" if mean_s < 0.05 else "12.5,200")
    out = {}
    for lam in [float(x) for x in rates.split(",")]:
        rng = np.random.default_rng(5)
        arr = np.cumsum(rng.exponential(1e9 / lam, nreq)).astype(np.int64)
        pidx = rng.integers(0, len(plans), nreq).astype(np.int32)
        gidx = np.zeros(nreq, np.int32)
        rec = {"offered_rps": lam, "offered_load": round(lam * mean_s, 3)}
        for mode in ("served", "fifo"):
            srv = gz.Server(max_inflight=args.inflight, max_batch=args.max_batch, heavy_ms=heavy_ms,
                            slow_share=args.slow_share)
            counts, lat, st = srv.replay(plans, [G], [1] * nreq, arr, pidx, gidx, fifo=(mode == "fifo"))
            srv.close()
            if [int(c) for c in counts] != [counts_alone[i] for i in pidx]:
                raise SystemExit(f"{mode} counts differ from counts alone")
            ms = np.sort(lat) / 1e6
            rec[mode] = {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                         "mean_ms": float(ms.mean()), "achieved_rps": st["achieved_rps"],
                         "max_queue": int(st["max_queue"]), "launches": int(st["launches"]),
                         "wall_s": st["wall_s"]}
        out[str(lam)] = rec
    lam0 = str(float(rates.split(",")[-1]))
    s = out[lam0]["served"]
    return _line("p99 latency, served (continuous batching)", s["p99_ms"], "ms", args, world,
                 1e3 * s["wall_s"] / nreq,
                 {"workload": f"Poisson stream of {nreq} requests per rate over {stream}, R-MAT scale "
                              f"{scale} ef 16 seed {scale} (+ oriented copy) resident; mix {names}",
                  "rates_per_s": rates},
                 hib=False, rates=out, service_alone=alone, stream_patterns=stream, heavy_ms=heavy_ms,
                 slow_share=args.slow_share or 0.75,
                 counts_alone=dict(zip(stream, counts_alone)), oracle_parity=parity)


def run_motifs(args, dist, world, rank, local):
    """Motif counting (Sec. 7.1-7.2, Table 2): every connected 3-, 4- and 5-vertex
    pattern counted on a seeded graph of the size of the paper's smallest dataset
    (ER with 3,264 vertices and ~4,536 edges, CiteSeer's counts; seed 7), and on
    R-MAT scale 12 ef 8 for a skewed one; each motif size as one merged program
    (gz_count_merged, the path of gz_count_motifs), against the same plans as
    separate programs in one batched call."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    graphs = {"er_citeseer_size": S.erdos_renyi(3264, 2 * 4536 / (3264 * 3263), 7),
              "rmat12_ef8": S.rmat(12, 8, 12)}
    res = {}
    total_ms = 0.0
    l0 = gz.kernel_launches()
    for gname, g in graphs.items():
        G = gz.Graph.from_csr(g).orient()
        for k in (3, 4, 5):
            # the same plans as one merged program and as separate programs in one
            # batched call; gz_count_motifs (planning included) must agree
            plans = [gz.Plan(a) for a in gz.motif_patterns(k)]
            counts, ms = _time_counts(lambda: gz.count_merged(plans, G, orientation=True), args.steps, stream)
            sep, ms_s = _time_counts(lambda: gz.count_batch(plans, [G] * len(plans), [True] * len(plans)),
                                     args.steps, stream)
            if sep != counts or gz.count_motifs(G, k, orientation=True) != counts:
                raise SystemExit(f"{gname} motif-{k}: merged and separate programs disagree")
            res[f"{gname}/motif{k}"] = {"patterns": len(counts), "sum": int(sum(counts)), **_summary(ms),
                                        "separate_programs_median_ms": round(statistics.median(ms_s), 4),
                                        "merged_speedup": round(statistics.median(ms_s) / statistics.median(ms), 3)}
            total_ms += statistics.median(ms)
    launches = gz.kernel_launches() - l0
    return _line("motif-3/4/5 count time, merged programs (sum of medians)", total_ms, "ms", args, world,
                 total_ms,
                 {"workload": "all connected 3-, 4- and 5-vertex patterns (2 + 6 + 21) on an ER graph "
                              "of CiteSeer's size (3,264 V, ~4,536 E, seed 7) and on R-MAT 12 ef 8",
                  "n_graphs": len(graphs)},
                 hib=False, motifs=res, gpu_launches=launches,
                 paper_context="Table 2: CiteSeer motif-3/4/5 in 0.9 / 2.4 / 38 ms on 2x8 Xeon cores")


SCHEDULE_PATTERNS = ["wedge", "path4", "star3", "c4", "paw", "diamond", "c5", "house", "hourglass",
                     "chordal5", "chordal6"]


def _r2_loglog(x, y):
    """R^2 of the least-squares line through (log x, log y)."""
    lx, ly = np.log(np.asarray(x, float)), np.log(np.asarray(y, float))
    if len(lx) < 3 or np.ptp(lx) == 0 or np.ptp(ly) == 0:
        return None
    r = np.corrcoef(lx, ly)[0, 1]
    return float(r * r)


def _spearman(x, y):
    if len(x) < 3:
        return None
    rx = np.argsort(np.argsort(x)).astype(float)
    ry = np.argsort(np.argsort(y)).astype(float)
    if np.ptp(rx) == 0 or np.ptp(ry) == 0:
        return None
    return float(np.corrcoef(rx, ry)[0, 1])


def run_schedules(args, dist, world, rank, local):
    """Measured schedule selection against the Sec. 5.4 performance model (the
    synthetic analogue of Fig. 11): every distinct schedule (Algorithm 4) of each
    pattern counts the whole oriented R-MAT graph (scale 14 ef 16 seed 14 by
    default) through gz_schedule_times; a schedule past --cutoff x the best is
    dropped. All kept schedules must give the same count. Reported per pattern:
    the model's pick and its time against the fastest, the rank correlation and
    the log-log R^2 of estimated cost against time."""
    import torch
    import paper_1911_12877_gb300 as gz
    import synthetic as S
    torch.cuda.set_device(local)
    scale = args.scale or 14
    g = S.rmat(scale, 16, scale)
    G = gz.Graph.from_csr(g).orient()
    names = args.patterns.split(",") if args.patterns else SCHEDULE_PATTERNS
    whole = [(0, g.n)]
    res, ratios, pooled = {}, [], ([], [])
    l0 = gz.kernel_launches()
    t0 = time.perf_counter()
    for name in names:
        a = gz.pattern_named(name)
        model = gz.Plan(a).info()["order"]
        times = gz.schedule_times(a, G, whole, orientation=True, cutoff=args.cutoff)
        kept = [t for t in times if t["ms"] >= 0]
        counts = {gz.count(gz.Plan(a, t["order"]), G, True) for t in kept}
        if len(counts) != 1:
            raise SystemExit(f"{name}: schedules disagree on the count: {sorted(counts)}")
        best = min(kept, key=lambda t: t["ms"])
        mt = next((t for t in times if t["order"] == model), None)
        if mt is None:
            raise SystemExit(f"{name}: the model's schedule {model} is not among Algorithm 4's")
        by_ms = sorted(kept, key=lambda t: t["ms"])
        rank_model = next((i + 1 for i, t in enumerate(by_ms) if t["order"] == model), None)
        r = {"schedules": len(times), "dropped": len(times) - len(kept), "count": counts.pop(),
             "model_order": model, "model_ms": round(mt["ms"], 3) if mt["ms"] >= 0 else None,
             "model_rank": rank_model, "best_order": best["order"], "best_ms": round(best["ms"], 3),
             "spearman_cost_vs_ms": _spearman([t["est_cost"] for t in kept], [t["ms"] for t in kept]),
             "r2_loglog_cost_vs_ms": _r2_loglog([t["est_cost"] for t in kept], [t["ms"] for t in kept])}
        # a dropped model schedule took at least cutoff x the best
        r["model_over_best"] = round((mt["ms"] if mt["ms"] >= 0 else args.cutoff * best["ms"]) / best["ms"], 3)
        ratios.append(r["model_over_best"])
        if len(kept) > 1:
            pooled[0].extend(t["est_cost"] for t in kept)
            pooled[1].extend(t["ms"] for t in kept)
        res[name] = r
    wall = time.perf_counter() - t0
    launches = gz.kernel_launches() - l0
    gm = float(np.exp(np.mean(np.log(ratios))))
    return _line("model-picked schedule time / fastest measured schedule (geometric mean)", gm, "x",
                 args, world, 1e3 * wall,
                 {"workload": f"every distinct schedule of {len(names)} patterns, whole-graph counts on "
                              f"R-MAT scale {scale} ef 16 seed {scale}, oriented; cutoff {args.cutoff}x"},
                 hib=False, patterns=res, gpu_launches=launches,
                 pooled_r2_loglog_cost_vs_ms=_r2_loglog(*pooled),
                 pooled_points=len(pooled[0]),
                 paper_context="Fig. 11: estimated against actual time, R^2 = 0.94 on Patents")


def run_planner(args, dist, world, rank, local):
    """Planner throughput on the host (Algorithm 4 schedules, Algorithm 1 +
    Theorem 2 restrictions, Sec. 5.4 model, program compile): every connected
    7-vertex pattern (853, Sec. 1) planned once per step, and K7 minus one edge
    (the Sec. 7.3 example). No GPU work."""
    import paper_1911_12877_gb300 as gz
    pats = gz.motif_patterns(7)
    for _ in range(args.warmup):
        for a in pats[:50]:
            gz.Plan(a)
    steps, worst = [], (0.0, None)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for i, a in enumerate(pats):
            t = time.perf_counter()
            gz.Plan(a)
            dt = time.perf_counter() - t
            if dt > worst[0]:
                worst = (dt, i)
        steps.append(time.perf_counter() - t0)
    k7e = []
    for _ in range(max(args.steps, 5)):
        t = time.perf_counter()
        gz.Plan("chordal7")
        k7e.append(time.perf_counter() - t)
    ms = 1e3 * statistics.median(steps)
    wa = pats[worst[1]]
    return _line("plan all 853 connected 7-vertex patterns", ms, "ms", args, world, ms,
                 {"workload": "host planner over every connected 7-vertex pattern, one thread"},
                 hib=False, gpu_launches=0,
                 max_pattern_ms=round(1e3 * worst[0], 3),
                 max_pattern_edges=int(wa.sum()) // 2,
                 max_pattern_schedules=len(gz.schedules(wa)),
                 k7_minus_edge_ms=round(1e3 * statistics.median(k7e), 3),
                 paper_context="Sec. 7.3: 853-pattern motif-7 compile 37 s; the hardest 7-vertex "
                               "patterns under 30 ms each; K7 minus one edge 0.6 ms (2x8 Xeon cores)")


EXTRA = {"triangle": run_triangle, "patterns": run_patterns, "pattern_samples": run_pattern_samples,
         "batched": run_batched,
         "served": run_served, "motifs": run_motifs, "schedules": run_schedules,
         "planner": run_planner}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gz", choices=["gz", "reference"])
    ap.add_argument("--config", default="clique",
                    choices=["clique", "triangle", "patterns", "pattern_samples", "batched", "served",
                             "motifs", "schedules", "planner"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-subconfigs", action="store_true",
                    help="skip the short triangle / patterns / batched records of the default run")
    ap.add_argument("--scale", type=int, default=0, help="R-MAT scale override (smaller cases)")
    ap.add_argument("--patterns", default="", help="patterns config: comma-separated subset")
    ap.add_argument("--cutoff", type=float, default=8.0,
                    help="schedules config: drop a schedule past this multiple of the best time")
    ap.add_argument("--full", default="", help="patterns config: patterns whose full count is timed "
                    "(default none at scale 22, all below)")
    ap.add_argument("--requests", type=int, default=0,
                    help="served config: requests per rate (0: 300 for millisecond requests, else about "
                         "60 s of service)")
    ap.add_argument("--rates", default="", help="served config: Poisson rates (default 12.5..200, or "
                                                "12.5,200 when requests take seconds)")
    ap.add_argument("--tune-min-ms", type=float, default=20.0,
                    help="batched config: queries taking at least this long alone are autotuned")
    ap.add_argument("--alone-cap", type=float, default=20.0,
                    help="served config: seconds a pattern may take alone before it is left out of the stream")
    ap.add_argument("--inflight", type=int, default=2, help="served config: concurrent launches")
    ap.add_argument("--max-batch", type=int, default=8, help="served config: requests per launch")
    ap.add_argument("--heavy-ms", type=float, default=0.0,
                    help="served config: slow-request threshold in ms (0: twice the median service time "
                         "alone, <0: off)")
    ap.add_argument("--slow-share", type=float, default=0.0,
                    help="served config: share of the device a slow request takes (0: library default 0.75)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "gz":
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        line = run_reference(args, world, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return 0
    import torch
    dist = init_dist(world, "nccl" if torch.cuda.is_available() else "gloo")
    if args.config == "clique":
        line = run_clique(args, dist, world, rank, local)
    else:
        line = EXTRA[args.config](args, dist, world, rank, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
