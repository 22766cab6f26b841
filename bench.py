#!/usr/bin/env python3
"""Throughput of balanced butterfly counting on GB300 (wedges/s).

One step = the whole path on one graph already resident in HBM: validation,
degree-priority ranking, sign-packed CSR build, work classification, wedge
aggregation and the C(.,2) reduction (bb_count_csr_device). The metric unit
is priority wedges (wedges u - v - w whose highest-priority vertex is an
endpoint; Algorithm 2 buckets exactly these) per second.

    python bench.py                       # 1 GPU, 2M x 500k Chung-Lu graph
    python bench.py --impl reference      # the CPU oracle, bounded samples
    torchrun --nproc-per-node N bench.py --gpus N   # N independent replicas

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "wedges/s"
UNIT = "wedges/s"
L2_FLUSH_BYTES = 512 << 20
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")

WORKLOADS = {
    "chunglu_2Mx500k_e20M_a2.1_p0.8": "chung_lu_2m",
    "vote_500x50000_p0.4_b2": "vote_500_50k",
    "uniform_2000x1000_e20000_p0.7": "uniform_2k_1k",
}
DEFAULT_WORKLOAD = "chunglu_2Mx500k_e20M_a2.1_p0.8"


def make_graph(name):
    from paper_2308_07932_gb300 import synth
    return getattr(synth, WORKLOADS[name])()


def priority_wedges(g) -> int:
    """Number of wedges u - v - w with u the highest-priority vertex of the
    three (Def. 4, ids u and |U|+v): per middle v and neighbour u ranked
    above v, the neighbours of v ranked below u. Sizes the reference arm's
    work in the metric's unit; computed on the host with NumPy sorts."""
    u, v, _ = g.edges()
    n = g.nU + g.nV
    deg = np.concatenate([np.diff(g.rowptr), np.bincount(g.col, minlength=g.nV)])
    order = np.lexsort((np.arange(n), deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    rs = np.concatenate([rank[u], rank[g.nU + v]])
    rd = np.concatenate([rank[g.nU + v], rank[u]])
    o = np.lexsort((rd, rs))
    rs, rd = rs[o], rd[o]
    pos = np.arange(rs.size) - np.searchsorted(rs, rs, side="left")
    return int(pos[rd > rs].sum())


# ------------------------------------------------------------ clock samples
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index: int, period_ms: int = 100):
        self.index, self.period_ms, self.proc = index, period_ms, None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", f"-lms={self.period_ms}"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) == len(self.FIELDS):
                self.rows.append(p)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------- CPU oracle
def oracle_rate(g, wedges: int, stride: int, offset: int, threads: int):
    """Times the oracle on every `stride`-th endpoint vertex (from `offset`)
    of its cheaper side and extrapolates to the full graph: the graph-view
    build is timed once (empty start list) and kept, the enumeration is
    scaled by full steps / sampled steps. Returns (wedges/s, seconds of the
    sampled call, description)."""
    import oracle
    from paper_2308_07932_gb300 import synth  # noqa: F401  (graph already built)
    degU = np.diff(g.rowptr)
    degV = np.bincount(g.col, minlength=g.nV)
    c2 = lambda d: (d.astype(np.float64) * (d - 1) / 2).sum()  # noqa: E731
    side = 1 if c2(degU) <= c2(degV) else 0     # endpoints on V when U-middles are cheaper
    n_side = g.nV if side == 1 else g.nU
    t0 = time.perf_counter()
    oracle.sample_count(g, np.zeros(0, np.int64), side, threads)
    t_view = time.perf_counter() - t0
    starts = np.arange(offset % stride, n_side, stride, dtype=np.int64)
    t0 = time.perf_counter()
    _, _, steps, full = oracle.sample_count(g, starts, side, threads)
    t_call = time.perf_counter() - t0
    t_enum = max(t_call - t_view, 1e-9)
    t_full = t_view + t_enum * (full / max(steps, 1))
    desc = (f"every {stride}th endpoint vertex of side {'UV'[side]} ({starts.size} of {n_side}), "
            f"{steps} of {full} two-hop steps; full-graph time extrapolated "
            f"{t_full:.1f} s (view build {t_view:.2f} s kept once)")
    return wedges / t_full, t_call, desc


def workload_config(name: str, g, wedges: int, world: int) -> dict:
    """The workload as both arms report it (identical keys and values)."""
    return {"workload": name, "nU": g.nU, "nV": g.nV, "nE": g.nE, "wedges": wedges,
            "inputs": "CSR resident in device memory when a timed GPU step starts",
            "l2": f"flushed before every timed GPU step ({L2_FLUSH_BYTES >> 20} MiB write, untimed)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    g = make_graph(args.workload)
    wedges = priority_wedges(g)
    threads = os.cpu_count() or 1
    # size each step at roughly 2-4 s of all-core work on this host
    stride = args.ref_stride
    for w in range(args.warmup):
        oracle_rate(g, wedges, stride, w, threads)
    rates, secs, desc = [], [], ""
    for k in range(args.steps):
        r, t, desc = oracle_rate(g, wedges, stride, args.warmup + k, threads)
        rates.append(r)
        secs.append(t)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic",
        "config": workload_config(args.workload, g, wedges, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"per step: {desc}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------- multi-rank helpers
def reduce_max(x: float, dist, device) -> float:
    """Max of x over all ranks (x itself when dist is None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, slowest_ms: float) -> float:
    """Units of all ranks per second of the slowest rank (replicas each do
    the same work, so the job ends with the slowest one)."""
    return world * units_per_rank / (slowest_ms / 1e3)


# ---------------------------------------------------------------- our path
def count_sha() -> str:
    h = hashlib.sha256()
    for f in ["count.cu", "walk.cuh", "graph.cuh", "common.cuh"]:
        with open(os.path.join(ROOT, "paper_2308_07932_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, workload: str):
    """ncu DRAM bytes per launch for `kernel` from profiles/traffic.json,
    or None when missing or taken on other kernel sources."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    e = rec.get(workload, {}).get(kernel)
    if not e or e.get("source_sha") != count_sha():
        return None
    return e.get("dram_bytes_per_launch")


def algorithmic_bytes(k: dict) -> int:
    """Bytes the wedge kernel must read by its definition: 4 per wedge (the
    packed entry of the suffix), 16 per middle (the anchor's entry, its
    suffix start, and the middle's two row offsets), 16 per anchor (row
    offsets and its work count); counters stay on chip."""
    return 4 * k["wedges"] + 16 * k["middles"] + 16 * k["anchors"]


def load_peaks():
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def load_bf16_peak():
    """Dense bf16 TFLOP/s for a kernel timed alone (the burst figure)."""
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(p["bf16_tflops"]), "measured"
    except (OSError, ValueError, KeyError):
        return 1900.0, "fallback"


def product_flops(g) -> int:
    """Floating-point operations of the matrix-product path's two GEMMs:
    X X^T and |X| |X|^T, each a x a over the padded width ld (a = the
    smaller side, ld = the other side rounded up to 8), 2 a^2 ld each."""
    a, b = min(g.nU, g.nV), max(g.nU, g.nV)
    ld = (b + 7) // 8 * 8
    return 2 * 2 * a * a * ld


def run_ours(args, world, rank, local_rank):
    import torch
    import paper_2308_07932_gb300 as pkg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    g = make_graph(args.workload)
    dev = torch.device("cuda", local_rank)
    rowptr = torch.from_numpy(g.rowptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    sign = torch.from_numpy(g.sign).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(local_rank)
    ctx.set_stream(stream.cuda_stream)
    ctx.set_timing(True)
    torch.cuda.synchronize()

    def step():
        return ctx.count_device(g.nU, g.nV, g.nE, rowptr.data_ptr(), col.data_ptr(),
                                sign.data_ptr())

    for _ in range(args.warmup):
        c = step()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    timings = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = pkg.launch_count()
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)          # L2 flush, outside the timed events
            ev[k][0].record(stream)
            c = step()
            ev[k][1].record(stream)
            timings.append(ctx.last_timing())
        torch.cuda.synchronize()
    launches = pkg.launch_count() - launches0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = reduce_max(sum(step_ms), dist, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(c.wedges, world, ms_per_step)

    # end to end through the public host-pointer call, pinned host inputs
    h_rowptr = torch.from_numpy(g.rowptr).pin_memory()
    h_col = torch.from_numpy(g.col).pin_memory()
    h_sign = torch.from_numpy(g.sign).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    ctx.set_timing(False)
    for _ in range(2):
        ctx.count_host_ptrs(g.nU, g.nV, g.nE, h_rowptr.data_ptr(), h_col.data_ptr(),
                            h_sign.data_ptr())
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ce = ctx.count_host_ptrs(g.nU, g.nV, g.nE, h_rowptr.data_ptr(), h_col.data_ptr(),
                                 h_sign.data_ptr())
    e2e_s = reduce_max((time.perf_counter() - t0) / e2e_steps, dist, dev)
    assert (ce.balanced, ce.total) == (c.balanced, c.total)

    # optional outputs on the resident graph: per-vertex (Algorithm 3's
    # quantity) and per-edge counts, each timed as one whole call
    opt = {}
    if rank == 0:
        res = ctx.upload(g)
        def timed(fn, reps=3):
            fn()
            best = None
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.fill_(1)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                out = fn()
                dt = (time.perf_counter() - t0) * 1e3
                best = dt if best is None else min(best, dt)
            return best, out
        opt["count_ms"], _ = timed(lambda: res.count())
        opt["count_per_vertex_ms"], cpv = timed(lambda: res.count(per_vertex=True))
        opt["count_per_edge_ms"], cpe = timed(lambda: res.count_edges())
        # every balanced butterfly has four vertices and four edges
        assert int(cpv.per_vertex.sum()) == 4 * c.balanced and int(cpe[0].sum()) == 4 * c.balanced
        # re-queries after sign flips: few flips take the incremental walk
        res.count()
        frng = np.random.default_rng(7)
        for k in (10, 1000, g.nE // 100):
            lists = iter([frng.choice(g.nE, k, replace=False) for _ in range(4)])
            ms, out = timed(lambda: res.count_flipped(next(lists)))
            opt[f"count_flipped_{k}_ms"] = ms
            opt[f"count_flipped_{k}_incremental"] = out[2]
        opt["timing"] = "host wall clock around the blocking call, best of 3, L2 flushed before"
        res.free()
        # the paper's baseline (BB-Base, Algorithm 1) against the bucket method,
        # on a 1.8 M-edge graph of the same recipe (BB-Base's work is the
        # number of butterflies, so the full graph would take seconds)
        from paper_2308_07932_gb300 import synth
        gb = synth.chung_lu_scaled(43, 2_000_000)
        rb = ctx.upload(gb)
        t_bucket, cb = timed(lambda: rb.count())
        t_base, bb_ = timed(lambda: rb.count_base(), reps=1)
        assert bb_ == (cb.balanced, cb.total)
        opt["base_vs_bucket"] = {"graph": gb.name, "edges": gb.nE, "butterflies": cb.total,
                                 "bucket_ms": t_bucket, "base_ms": t_base,
                                 "base_over_bucket": t_base / t_bucket}
        rb.free()

    # dominant wedge kernel and its roofline
    kern = kernel_table(pkg, timings)
    build_ms = statistics.mean(t["build_ms"] for t in timings)
    count_ms = statistics.mean(t["count_ms"] for t in timings)
    top = max(kern, key=lambda k: kern[k]["ms"])
    peak, peak_kind = load_peaks()
    ach = algorithmic_bytes(kern[top]) / (kern[top]["ms"] / 1e3) / 1e9 if kern[top]["ms"] else 0.0
    product_ms = statistics.mean(t["product_ms"] for t in timings)
    clocks = clk.summary()
    # second ceiling: shared-memory atomic throughput (one atomic per wedge)
    atomics = {w: pkg.probe_shared_atomics(local_rank, w) for w in (2048, 49152)}
    count_rate = c.wedges / (count_ms / 1e3)
    if product_ms > 0:  # counted by the matrix-product path (tensor-bound)
        tpeak, tkind = load_bf16_peak()
        tach = product_flops(g) / (product_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "kernel": "matrix product (fill, GEMMs, pair sums)",
                    "achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
                    "peak_kind": tkind, "flops": product_flops(g), "traffic": None}
    else:
        roofline = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_kind": peak_kind,
                    "algorithmic_bytes": algorithmic_bytes(kern[top]),
                    "traffic": traffic_for(top, args.workload),
                    "atomic_ceiling": {
                        "unit": "shared-memory atomics/s (one per wedge)",
                        "window_2048": atomics[2048], "window_49152": atomics[49152],
                        "count_phase_wedges_per_s": count_rate,
                        "frac": count_rate / atomics[2048]}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
        "config": workload_config(args.workload, g, c.wedges, world),
        "counts": {"balanced": c.balanced, "total": c.total},
        "phases_ms": {"build": build_ms, "count": count_ms, "matrix_product": product_ms,
                      **{k: v["ms"] for k, v in kern.items()}},
        "kernels": kern,
        "roofline": roofline,
        "e2e": {"value": whole_job_rate(c.wedges, world, e2e_s * 1e3), "unit": UNIT,
                "h2d_bytes_per_step": g.rowptr.nbytes + g.col.nbytes + g.sign.nbytes,
                "d2h_bytes_per_step": 52},
        "gpu_launches": launches,
        "clocks": clocks,
        "optional_outputs": opt,
    }
    if rank == 0 and world == 1 and not args.no_extra_workloads:
        line["workloads"] = {w: run_workload_leg(args, w, local_rank)
                             for w in EXTRA_WORKLOADS if w != args.workload}
    if rank == 0 and world == 1 and args.batch_graphs > 0:
        line["batch"] = run_batch_leg(args, local_rank)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serving"] = run_serve_leg(args, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, secs, desc = oracle_rate(g, c.wedges, args.cpu_stride, 0, os.cpu_count() or 1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count() or 1,
                                "kind": "oracle", "sample": desc, "seconds": secs}
        r1, s1, d1 = oracle_rate(g, c.wedges, args.cpu_stride * 16, 0, 1)
        line["cpu_baseline"]["single_thread"] = {"value": r1, "cores": 1, "sample": d1,
                                                 "seconds": s1}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------ the other single graphs
EXTRA_WORKLOADS = ["vote_500x50000_p0.4_b2", "uniform_2000x1000_e20000_p0.7"]


def kernel_table(pkg, timings):
    """Per wedge kernel: mean CUDA-event time over the timed steps and its
    work (wedges, middles, anchors)."""
    return {k: {"ms": statistics.mean(t["kernels"][k]["ms"] for t in timings),
                **{f: timings[-1]["kernels"][k][f] for f in ("wedges", "middles", "anchors")}}
            for k in pkg.KERNELS}


def run_workload_leg(args, name: str, dev_index: int) -> dict:
    """One more single-graph configuration, measured like the headline: the
    whole path through bb_count_csr_device on the device-resident graph (L2
    flushed before each step, CUDA events), the dominant kernel's roofline,
    the same through bb_count_csr from pinned host buffers (e2e), and the
    oracle on the host cores. The 500 x 50k vote graph stands in for the
    dense vote-like datasets; the 2k x 1k uniform graph is launch-bound, so
    its figure is the latency of one call."""
    import torch
    import paper_2308_07932_gb300 as pkg

    g = make_graph(name)
    dev = torch.device("cuda", dev_index)
    t_rp, t_cl, t_sg = (torch.from_numpy(a).to(dev) for a in (g.rowptr, g.col, g.sign))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(dev_index)
    ctx.set_stream(stream.cuda_stream)
    ctx.set_timing(True)
    torch.cuda.synchronize()

    def step():
        return ctx.count_device(g.nU, g.nV, g.nE, t_rp.data_ptr(), t_cl.data_ptr(),
                                t_sg.data_ptr())

    for _ in range(max(3, args.warmup)):
        c = step()
    steps = max(5, args.extra_steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    timings = []
    with ClockSampler(dev_index) as clk:
        for k in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            c = step()
            ev[k][1].record(stream)
            timings.append(ctx.last_timing())
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    ms_step = statistics.mean(ms)
    kern = kernel_table(pkg, timings)
    top = max(kern, key=lambda k: kern[k]["ms"])
    peak, peak_kind = load_peaks()
    ach = algorithmic_bytes(kern[top]) / (kern[top]["ms"] / 1e3) / 1e9 if kern[top]["ms"] else 0.0
    product_ms = statistics.mean(t["product_ms"] for t in timings)
    if product_ms > 0:
        # counted by the matrix-product path: its roofline is the bf16 tensor
        # rate (fill, both GEMMs and the pair sums inside the timed span)
        tpeak, tkind = load_bf16_peak()
        tach = product_flops(g) / (product_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "kernel": "matrix product (fill, GEMMs, pair sums)",
                    "achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
                    "peak_kind": tkind, "flops": product_flops(g), "traffic": None}
    else:
        roofline = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": peak,
                    "unit": "GB/s", "frac": ach / peak, "peak_kind": peak_kind,
                    "algorithmic_bytes": algorithmic_bytes(kern[top]),
                    "traffic": traffic_for(top, name)}
    # end to end from pinned host buffers
    h = [torch.from_numpy(a).pin_memory() for a in (g.rowptr, g.col, g.sign)]
    ctx.set_timing(False)
    for _ in range(2):
        ctx.count_host_ptrs(g.nU, g.nV, g.nE, *(x.data_ptr() for x in h))
    e2e = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ce = ctx.count_host_ptrs(g.nU, g.nV, g.nE, *(x.data_ptr() for x in h))
        e2e.append(time.perf_counter() - t0)
    assert (ce.balanced, ce.total) == (c.balanced, c.total)
    ctx.close()
    e2e_s = statistics.mean(e2e)
    cores = os.cpu_count() or 1
    rate, secs, desc = oracle_rate(g, c.wedges, args.cpu_stride if g.nE > 1e6 else 1, 0, cores)
    return {
        "metric": METRIC, "unit": UNIT, "value": c.wedges / (ms_step / 1e3),
        "ms_per_step": ms_step, "steps": steps,
        "latency_ms": {"device_median": statistics.median(ms),
                       "e2e_median": 1e3 * statistics.median(e2e)},
        "config": workload_config(name, g, c.wedges, 1),
        "counts": {"balanced": c.balanced, "total": c.total},
        "phases_ms": {"build": statistics.mean(t["build_ms"] for t in timings),
                      "count": statistics.mean(t["count_ms"] for t in timings),
                      "matrix_product": product_ms,
                      **{k: v["ms"] for k, v in kern.items()}},
        "kernels": kern,
        "roofline": roofline,
        "e2e": {"value": c.wedges / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": g.rowptr.nbytes + g.col.nbytes + g.sign.nbytes,
                "d2h_bytes_per_step": 52},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc, "seconds": secs},
        "clocks": clk.summary(),
    }


# ------------------------------------------------------- batched counting
BATCH_GRAPHS = 4096


def run_batch_leg(args, dev_index: int) -> dict:
    """Many-graph leg: the batched mix (graph i seeded 4+i; |E| log-uniform in
    [1e3, 2e6], |U|:|V| in [1, 10], exponent in [2.1, 2.8], p(+) in [0.5,
    0.9]) uploaded once, then every graph counted per step, two ways: one
    batched launch sequence (class-queue kernels, captured CUDA graph, shapes
    from the autotuner) and one bb_count per graph. Both give identical
    counts (checked); graphs/s is graphs per second of device time."""
    import torch
    import paper_2308_07932_gb300 as pkg
    from paper_2308_07932_gb300 import synth

    n = args.batch_graphs
    t0 = time.perf_counter()
    hosts = synth.batch_graphs(n)
    gen_s = time.perf_counter() - t0
    dev = torch.device("cuda", dev_index)
    stream = torch.cuda.Stream(device=dev)
    ctx = pkg.Context(dev_index)
    ctx.set_stream(stream.cuda_stream)
    t0 = time.perf_counter()
    graphs = [ctx.upload(g) for g in hosts]
    upload_s = time.perf_counter() - t0
    edges = sum(g.nE for g in hosts)
    wedges = sum(g.info()[3] for g in graphs)
    del hosts
    batch = pkg.Batch(ctx, graphs)
    tune, tune_ms = batch.autotune(reps=3)
    bal, tot = batch.count()                     # capture + first replay
    for _ in range(args.warmup):
        batch.count()
    launches0 = pkg.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.batch_steps)]
    wall0 = time.perf_counter()
    with ClockSampler(dev_index) as clk:
        for k in range(args.batch_steps):
            ev[k][0].record(stream)
            b2, t2 = batch.count()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    wall = (time.perf_counter() - wall0) / args.batch_steps
    launches = pkg.launch_count() - launches0
    assert (b2 == bal).all() and (t2 == tot).all()
    ms = statistics.median(a.elapsed_time(b) for a, b in ev)
    # one traced count: each class kernel's time (uncaptured, serial)
    ctx.set_timing(True)
    b3, t3 = batch.count()
    tr = ctx.last_timing()
    ctx.set_timing(False)
    assert (b3 == bal).all() and (t3 == tot).all()
    classes = {k: dict(tr["kernels"][k]) for k in pkg.KERNELS}
    # one bb_count per graph, on the same resident graphs
    per_ms = []
    for k in range(max(1, args.batch_single_steps) + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        single = [g.count() for g in graphs]
        e1.record(stream)
        torch.cuda.synchronize()
        if k > 0:                                 # first pass is a warm-up
            per_ms.append(e0.elapsed_time(e1))
    assert [(c.balanced, c.total) for c in single] == list(zip(bal.tolist(), tot.tolist()))
    single_ms = statistics.median(per_ms)
    batch.free()
    for g in graphs:
        g.free()
    ctx.close()
    return {
        "graphs": n, "edges": edges, "wedges": wedges,
        "graphs_per_s": n / (ms / 1e3), "wedges_per_s": wedges / (ms / 1e3), "ms_per_step": ms,
        "wall_ms_per_step": wall * 1e3, "steps": args.batch_steps,
        "per_graph_launches": {"graphs_per_s": n / (single_ms / 1e3), "ms_per_step": single_ms,
                               "steps": len(per_ms)},
        "speedup_vs_per_graph": single_ms / ms,
        "traced_classes": classes, "traced_count_ms": tr["count_ms"],
        "tune": tune.to_dict(), "tune_ms": tune_ms, "gpu_launches": launches,
        "setup_s": {"generate": gen_s, "upload_and_build": upload_s},
        "l2": "working set larger than L2 (no flush needed)" if edges * 13 > 256e6
              else "working set may fit L2 (not flushed)",
        "clocks": clk.summary(),
    }


# ------------------------------------------------------------------ serving
SERVE_BUDGET = 120 << 30


def serve_trace(n_req: int, rate: float, pool_n: int, seed: int, requery: float = 0.2,
                flip_frac: float = 0.01):
    """Poisson arrivals at `rate` req/s. A request is a re-query (probability
    `requery`, once some graph was requested) of a random earlier key with
    `flip_frac` of its edge signs flipped, else a new key whose graph is the
    next pool graph (pool graphs repeat under new keys once used up)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    reqs, keys = [], []
    for k in range(n_req):
        if keys and rng.random() < requery:
            key = keys[int(rng.integers(len(keys)))]
            reqs.append((float(t[k]), key, None, float(rng.random())))
        else:
            key = len(keys) + 1
            keys.append(key)
            reqs.append((float(t[k]), key, (key - 1) % pool_n, None))
    return reqs


def flip_list(nE: int, frac: float, u: float):
    """Deterministic flip list for a re-query: `frac` of the edges, seeded by u."""
    rng = np.random.default_rng(int(u * 2**31))
    return rng.choice(nE, size=max(1, int(nE * frac)), replace=False)


def pctl(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if xs else None


def run_serve_leg(args, dev_index: int) -> dict:
    """Request-loop leg: graphs drawn as the 2M x 500k workload at |E|
    log-uniform in [1e4, 5e7], Poisson arrivals at each swept rate, 20%
    re-queries of a resident graph with 1% of its edge signs flipped, a
    120 GiB HBM budget. Served = the engine (4 slots, managed cache in a
    120 GiB arena); plain = per request upload + count + free, one at a
    time. Every request (flip lists included) is generated before the trace
    starts, and each path is warmed up on graphs outside the trace. Latency
    = arrival to the moment the client holds the result, on the client's
    clock for both paths; both paths must agree on every count."""
    import paper_2308_07932_gb300 as pkg
    from concurrent.futures import ThreadPoolExecutor
    from paper_2308_07932_gb300 import synth

    t0 = time.perf_counter()
    with ThreadPoolExecutor(min(32, os.cpu_count() or 4)) as ex:
        pool = list(ex.map(synth.serving_graph, range(args.serve_pool)))
        warm = list(ex.map(synth.serving_graph, range(10_000, 10_004)))
    gen_s = time.perf_counter() - t0
    rates = [float(x) for x in args.serve_rates.split(",")]
    out = {"pool_graphs": len(pool), "pool_edges": int(sum(g.nE for g in pool)),
           "requests_per_rate": args.serve_requests, "slots": args.serve_slots,
           "budget_bytes": SERVE_BUDGET, "setup_s": {"generate": gen_s},
           "latency": "arrival to result held by the client, client clock, both paths",
           "warmup": f"{len(warm)} graphs outside the trace through each path before it",
           "rates": []}

    for ri, rate in enumerate(rates):
        trace = serve_trace(args.serve_requests, rate, len(pool), seed=100 + ri)
        # resolve every request before the clock starts: graph, flip list and
        # the key's signs before and after it. A re-query carries the CSR with
        # the signs before its flips: the engine ignores it while the key is
        # resident and uploads it when the key was evicted meanwhile.
        key_graph, state, reqs = {}, {}, []
        for at, key, gidx, u in trace:
            if gidx is not None:
                key_graph[key] = gidx
                state[key] = pool[gidx].sign
                reqs.append((at, key, gidx, None, pool[gidx], pool[gidx]))
            else:
                g0 = pool[key_graph[key]]
                fl = flip_list(g0.nE, 0.01, u)
                pre = state[key]
                post = pre.copy()
                post[fl] = -post[fl]
                state[key] = post
                mk = lambda sg: synth.SignedBipartite(g0.nU, g0.nV, g0.rowptr, g0.col, sg, g0.name)  # noqa: E731
                reqs.append((at, key, key_graph[key], fl, mk(pre), mk(post)))
        del state
        # ---- served
        ctx = pkg.Context(dev_index, budget_bytes=SERVE_BUDGET + (4 << 30))
        ctx.serve(slots=args.serve_slots, arena_bytes=SERVE_BUDGET)
        for k, g in enumerate(warm):
            ctx.submit_request(1_000_000 + k, g).wait()
        lat, got, pending = [0.0] * len(reqs), [None] * len(reqs), []
        start = time.perf_counter()
        i = 0
        with ClockSampler(dev_index) as clk:
            while i < len(reqs) or pending:
                now = time.perf_counter() - start
                busy = False
                while i < len(reqs) and reqs[i][0] <= now:
                    at, key, gidx, fl, pre, _ = reqs[i]
                    tk = ctx.submit_request(key, pre, fl)
                    pending.append((i, tk))
                    i += 1
                    busy = True
                still = []
                for j, tk in pending:
                    r = tk.poll()
                    if r is None:
                        still.append((j, tk))
                    else:
                        lat[j] = (time.perf_counter() - start - reqs[j][0]) * 1e3
                        got[j] = (r.balanced, r.total)
                        busy = True
                pending = still
                if not busy:
                    time.sleep(50e-6)
        served_s = time.perf_counter() - start
        stats = ctx.serve_stats()
        ctx.close()
        # ---- plain: upload + count + free per request, one at a time
        ctx = pkg.Context(dev_index, budget_bytes=SERVE_BUDGET)
        for g in warm:
            gr = ctx.upload(g)
            gr.count()
            gr.free()
        plat, pgot = [0.0] * len(reqs), [None] * len(reqs)
        start = time.perf_counter()
        for j, (at, key, gidx, fl, _, post) in enumerate(reqs):
            now = time.perf_counter() - start
            if now < at:
                time.sleep(at - now)
            gr = ctx.upload(post)
            c = gr.count()
            gr.free()
            pgot[j] = (c.balanced, c.total)
            plat[j] = (time.perf_counter() - start - at) * 1e3
        plain_s = time.perf_counter() - start
        ctx.close()
        assert got == pgot, "served and plain counts differ"
        out["rates"].append({
            "rate_req_s": rate,
            "served": {"graphs_per_s": len(reqs) / served_s, "p50_ms": pctl(lat, 50),
                       "p99_ms": pctl(lat, 99), "max_ms": max(lat),
                       "cache_hits": stats["cache_hits"], "uploads": stats["uploads"],
                       "evictions": stats["evictions"], "clocks": clk.summary()},
            "plain": {"graphs_per_s": len(reqs) / plain_s, "p50_ms": pctl(plat, 50),
                      "p99_ms": pctl(plat, 99), "max_ms": max(plat)},
        })
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-stride", type=int, default=8,
                    help="oracle sample: every k-th endpoint vertex")
    ap.add_argument("--wedge-path", action="store_true",
                    help="count every graph with the wedge kernels (no matrix-product path)")
    ap.add_argument("--no-extra-workloads", action="store_true",
                    help="skip the vote 500x50k and uniform 2k x 1k legs")
    ap.add_argument("--extra-steps", type=int, default=20,
                    help="timed steps of each extra single-graph leg")
    ap.add_argument("--batch-graphs", type=int, default=BATCH_GRAPHS,
                    help="graphs in the batched leg (0 = skip the leg)")
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-single-steps", type=int, default=2)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="requests per rate in the serving leg (0 = skip the leg)")
    ap.add_argument("--serve-rates", default="50,200,400,800", help="arrival rates, req/s")
    ap.add_argument("--serve-pool", type=int, default=24)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--ref-stride", type=int, default=64,
                    help="reference arm: every k-th endpoint vertex per step")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        if args.wedge_path:
            import paper_2308_07932_gb300 as pkg
            pkg.set_matrix_product(False)
        run_ours(args, world, rank, local_rank)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
