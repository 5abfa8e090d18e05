#!/usr/bin/env python3
"""Benchmark of the projected-Krylov verification path on GB300.

One *step* is one whole verification query of the workload (initial vector,
krylov_m Lanczos iterations with the on-the-fly output projection, the batched
exponential for every time step, the bounds and the first-violation scan).

Default workload: 3D heat on a 1000^3 grid (n = 1e9), 7-point matrix-free
Laplacian, Dirichlet-0, coefficient 0.01, h = 1/1001, a 100^3 heated corner
block (one generator, u in [0.9, 1.1]), centre-cell output, dt = 0.02,
200 steps, Lanczos m = 30.

metric: Lanczos-step GB/s = algorithmic bytes of the Lanczos iterations
(read v_j, read v_{j-1}, write v_{j+1}: 3 vectors of n elements per
iteration) / time per query.  The vectors (8 GB FP64, 4 GB FP32) are far
larger than the 126 MB L2, so no flush is needed between iterations.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "Lanczos-step HBM GB/s (1e9-dim heat); queries/s + p99 at <=1e-6 rel bound error"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(name: str, precision: str):
    if name == "heat3d-1000":
        return W.heat3d_1000(precision=precision)
    if name == "heat3d-100":
        return W.heat3d_100(precision=precision)
    if name == "heat2d-20":
        return W.heat2d_20(precision=precision)
    if name == "heat3d-512":
        # profiling case: 1.6 GB of FP32 vectors (above L2, a few GB on the
        # device), few launches before the captured ones
        return W.heat((512, 512, 512), block=(50, 50, 50), output="centre", dt=0.02, steps=10, m=4,
                      precision=precision, name="heat3d-512^3-profile")
    raise ValueError(name)


def bytes_per_iteration(p) -> float:
    es = 8 if p.precision == "fp64" else 4
    return 3.0 * es * p.system.n


# ----------------------------------------------------------------- clocks
CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def summarize_clocks(samples, t0=None, t1=None):
    """Median SM clock, max clock and active throttle reasons of nvidia-smi
    lines "index, sm, max_sm, power, hw, hw_thermal, sw_thermal, sw_power_cap"
    taken at host times t; only samples inside [t0, t1] count when the window
    holds any (a short timed region may fall between two samples, then the
    nearest ones are used)."""
    parsed = []
    for t, ln in samples:
        parts = [x.strip() for x in ln.split(",")]
        if len(parts) < 8:
            continue
        try:
            sm, mx = float(parts[1]), float(parts[2])
        except ValueError:
            continue
        reasons = {nm for nm, v in zip(CLOCK_REASONS, parts[4:8]) if v.lower() == "active"}
        parsed.append((t, sm, mx, reasons))
    if not parsed:
        return None
    inside = [s for s in parsed if (t0 is None or s[0] >= t0) and (t1 is None or s[0] <= t1)]
    if not inside and t0 is not None and t1 is not None:
        mid = 0.5 * (t0 + t1)
        inside = sorted(parsed, key=lambda s: abs(s[0] - mid))[:2]
    if not inside:
        inside = parsed
    return {"sm_mhz": statistics.median(s[1] for s in inside), "sm_max_mhz": max(s[2] for s in inside),
            "reasons": sorted(set().union(*(s[3] for s in inside))), "samples": len(inside)}


class ClockSampler:
    """nvidia-smi sampling (200 ms) around the timed region: start() waits for
    the first sample, mark() brackets the timed region on the host clock."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.samples: list[tuple[float, str]] = []
        self.window = [None, None]

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t_end = time.perf_counter() + 3.0
        while not self.samples and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def mark(self, which: int):
        self.window[which] = time.perf_counter()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)  # one more sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.samples, *self.window)


def reduce_max(x: float, world: int, device: str = "cuda") -> float:
    """Max of a per-rank value over all ranks (the slowest replica sets the
    whole job's time); identity at world = 1."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job rate of `world` replicas that each process units_per_rank
    units, timed by the slowest one."""
    return world * units_per_rank / (ms_max * 1e-3)


# ------------------------------------------------------------ CPU baseline
def cpu_baseline(p, iters: int = 4):
    """The oracle's Lanczos (Alg. 3/4, plain FP64 C with OpenMP) on the same
    grid for a bounded number of iterations; same byte model as the GPU."""
    import oracle
    n = p.system.n
    e = W.column_dense(p.columns[0], n, p.system.dims)
    b0 = float(np.sqrt(np.dot(e, e)))
    e /= b0
    t0 = time.perf_counter()
    oracle.krylov(p.system, e, iters, p.C_row_ptr, p.C_col, p.C_val, method="lanczos")
    t = time.perf_counter() - t0
    del e
    gbs = iters * 3.0 * 8 * n / t / 1e9
    cores = oracle.num_threads()
    # the same on one thread, a shorter sample
    one = max(1, iters // 12)
    oracle.set_threads(1)
    try:
        e = W.column_dense(p.columns[0], n, p.system.dims)
        e /= b0
        t0 = time.perf_counter()
        oracle.krylov(p.system, e, one, p.C_row_ptr, p.C_col, p.C_val, method="lanczos")
        t1 = time.perf_counter() - t0
        del e
    finally:
        oracle.set_threads(cores)
    return {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{iters} Lanczos iterations of the FP64 oracle on the full {p.name} grid "
                      f"(n={n}), {t:.1f} s",
            "single_thread": {"value": one * 3.0 * 8 * n / t1 / 1e9, "unit": "GB/s", "cores": 1,
                              "sample": f"{one} iterations, {t1:.1f} s"}}


# ------------------------------------------------------------------ GPU arm
GRID_KERNELS = ["lanczos_fused", "lanczos_fused64", "stencil_update", "stencil_alpha", "stencil_init", "expm_per_step",
                "expm_propagate", "bounds", "bounds_finish"]


def fp64_instr_per_launch(p) -> float:
    """Algorithmic FP64 instructions of one single-pass FP64 iteration: the
    update stored as w / (s_j kappa_x) = (l + r) + ry (d + u) + rz (m + p)
    + rc c + ra a takes 3 pair sums and 4 fused multiply-adds a grid point (3
    FMAs in the first iteration, which has no v_{j-1}); averaged over a
    query's m launches."""
    return p.system.n * (6.0 + 7.0 * (p.m - 1)) / p.m


def time_query(ctx, ph, stream, steps: int, warmup: int, torch, barrier=None, clocks=None):
    """Device time of `steps` enqueues of one query (CUDA events on the
    library stream) with per-kernel times from the library's own events."""
    for _ in range(warmup):
        ph.enqueue()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ctx.profile_enable(True)
    if clocks:
        clocks.start()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.mark(0)
    ev0.record(stream)
    for _ in range(steps):
        ph.enqueue()
    ev1.record(stream)
    torch.cuda.synchronize()
    if clocks:
        clocks.mark(1)
    if barrier:
        barrier()
    clk = clocks.stop() if clocks else None
    ms_total = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    kern = {}
    for name in GRID_KERNELS:
        nl, tms = ctx.profile_read(name)
        if nl:
            kern[name] = (nl, tms)
    ctx.profile_enable(False)
    return ms_total, kern, launches, clk


FP64_NOMINAL_TIPS = 0.625  # nominal FP64 rate of the part, T instructions/s (1.25 TFLOP/s dense)


def roofline(dom: str, kern: dict, p, fp64_peak: float) -> dict:
    """Roofline of the dominant kernel: algorithmic work per launch over its
    average launch time (library events), against the measured peak."""
    nl, tms = kern[dom]
    avg_s = tms / nl * 1e-3
    bpi = bytes_per_iteration(p)
    hbm_peak, hbm_kind = peaks()
    if dom == "lanczos_fused64":
        instr = fp64_instr_per_launch(p)
        ach = instr / avg_s / 1e12
        pk = fp64_peak / 1e12
        return {"bound": "alu", "kernel": dom, "achieved": ach, "peak": pk, "unit": "T FP64-instr/s",
                "frac": ach / pk,
                "peak_kind": "measured in this run: kv_diag_fp64_rate (FP64 FMA chains on every SM, best of 5, "
                             "CUDA events)",
                "peak_nominal": FP64_NOMINAL_TIPS, "frac_nominal": ach / FP64_NOMINAL_TIPS,
                "peak_nominal_kind": "1.25 TFLOP/s dense FP64 (the part's nominal figure) = 0.625 T FP64 "
                                     "instructions/s (one FMA, add or multiply each)",
                "algorithmic_fp64_instr_per_launch": instr, "avg_launch_ms": avg_s * 1e3,
                "algorithmic_bytes_per_launch": bpi, "hbm_achieved_gbs": bpi / avg_s / 1e9,
                "hbm_frac": bpi / avg_s / 1e9 / hbm_peak, "traffic": profiled_traffic(dom, p)}
    alg = {"lanczos_fused": bpi, "stencil_update": bpi, "stencil_alpha": bpi / 3.0}.get(dom)
    ach = alg / avg_s / 1e9 if alg else None
    return {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
            "frac": (ach / hbm_peak) if ach else None, "peak_kind": hbm_kind + " (copy, burst)",
            "algorithmic_bytes_per_launch": alg, "avg_launch_ms": avg_s * 1e3, "traffic": profiled_traffic(dom, p)}


def run_gpu(args, rank: int, world: int):
    import torch
    import paper_1804_01583_gb300 as kv
    from paper_1804_01583_gb300 import build as kvbuild

    kvbuild.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    fp64_peak, fp64_add = kv.diag_fp64_rate(dev)
    p = workload(args.workload, args.precision)
    pool_bytes = max(kv_bytes_guess(p), 1 << 30)
    stream = torch.cuda.Stream()
    ctx = kv.Context(pool_bytes, device=dev, stream=stream)
    sysh = kv.System(ctx, p.system, p.precision)
    ph = kv.ProblemHandle(ctx, sysh, p, expm_mode=args.expm)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    ms_total, kern, launches, clk = time_query(ctx, ph, stream, args.steps, args.warmup, torch, barrier,
                                               ClockSampler(dev))
    res = ph.fetch(full=False)
    ph.close()
    sysh.close()
    ms_step = reduce_max(ms_total / args.steps, world)
    bpi = bytes_per_iteration(p)
    gbs = replica_throughput(p.m * bpi, ms_step, world) / 1e9

    # end to end through the public API with host inputs: system + problem
    # creation (host -> device), run, result fetch (device -> host)
    e2e_ms = []
    for q in range(max(2, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = kv.System(ctx, p.system, p.precision)
        h2 = kv.ProblemHandle(ctx, s2, p, expm_mode=args.expm)
        out = h2.run(full=False)
        t1 = time.perf_counter()
        h2.close()
        s2.close()
        if q > 0:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e = reduce_max(statistics.median(e2e_ms), world)
    h2d = 8 * (p.o + 1) + 8 * len(p.C_col) * 2 + 8 * p.o + 16 * p.i + 64 * p.i
    d2h = 8 * 2 * p.o * (p.steps + 1) + 8 * p.i + 16
    out_e2e = {"value": replica_throughput(p.m * bpi, e2e, world) / 1e9, "unit": "GB/s", "ms_per_step": e2e,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    dom = max(kern, key=lambda k: kern[k][1])
    kernels = {k: {"launches": v[0], "avg_ms": v[1] / v[0], "share": v[1] / ms_total} for k, v in kern.items()}
    line = {
        "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if p.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": p.name, "n": p.system.n, "krylov_m": p.m, "steps_per_query": p.steps,
                   "precision": p.precision, "expm": args.expm, "l2": "inputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}",
                   "bytes_per_point_per_iteration": 3 * (8 if p.precision == "fp64" else 4)},
        "queries_per_s": world * 1e3 / ms_step,
        "roofline": roofline(dom, kern, p, fp64_peak), "kernels": kernels, "e2e": out_e2e,
        "gpu_launches": launches, "clocks": clk, "first_violation_step": res["viol_step"],
        "lemma1_bound": float(res["err_bound"][0]),
        "fp64_rate": {"fma_per_s": fp64_peak, "add_per_s": fp64_add, "sms": torch.cuda.get_device_properties(dev)
                      .multi_processor_count},
    }
    if args.compare_fp64:
        other = "fp32" if p.precision == "fp64" else "fp64"
        sub = time_other_precision(kv, ctx, args, other, torch, stream, fp64_peak)
        sub["speedup_over_fp64" if other == "fp32" else "speedup_of_fp32"] = (
            ms_step / sub["ms_per_step"] if other == "fp32" else sub["ms_per_step"] / ms_step)
        line["fp32_storage" if other == "fp32" else "fp64_plain"] = sub
    ctx.close()
    return line, p


def time_other_precision(kv, ctx, args, precision, torch, stream, fp64_peak):
    """The same query in the other storage precision on the same context, with
    its own kernel times and roofline."""
    q = workload(args.workload, precision)
    sysh = kv.System(ctx, q.system, q.precision)
    try:
        ph = kv.ProblemHandle(ctx, sysh, q, expm_mode=args.expm)
    except kv.KvError as e:
        sysh.close()
        return {"skipped": str(e)}
    k = max(2, args.steps)
    ms_total, kern, launches, _ = time_query(ctx, ph, stream, k, max(1, args.warmup), torch)
    ph.close()
    sysh.close()
    ms = ms_total / k
    dom = max(kern, key=lambda x: kern[x][1])
    return {"precision": precision, "dtype": "f32" if precision == "fp32" else "f64", "ms_per_step": ms,
            "value": q.m * bytes_per_iteration(q) / (ms * 1e-3) / 1e9, "unit": "GB/s", "steps": k,
            "bytes_per_point_per_iteration": 3 * (8 if precision == "fp64" else 4),
            "roofline": roofline(dom, kern, q, fp64_peak),
            "kernels": {x: {"launches": v[0], "avg_ms": v[1] / v[0], "share": v[1] / ms_total}
                        for x, v in kern.items()}, "gpu_launches": launches}


def profiled_traffic(kernel: str, p):
    """DRAM bytes per launch from the committed ncu summary of this kernel, if
    the kernel source has not changed since the capture (hash match), scaled
    from the captured grid to this one by the number of points."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{kernel}.json")
    try:
        with open(path) as f:
            d = json.load(f)
        src = os.path.join(ROOT, d["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if h != d["source_sha256"] or d.get("precision") != p.precision:
            return None
        return d["dram_bytes_per_launch"] * p.system.n / d["n"]
    except Exception:
        return None


SERVE_KINDS = ("heat2d", "heat3d", "csr")


def serve_kind(q) -> str:
    return next(k for k in SERVE_KINDS if f"-{k}" in q.name)


def serve_oracle_sample(qs, per_kind: int = 6, seed: int = 7):
    """Queries whose served results the CPU leg compares with the oracle:
    `per_kind` of each kind, drawn with a seed among those the oracle runs in
    about a second on the host (heat grids up to 250^3 points, CSR systems up
    to 5e5 rows)."""
    rng = np.random.default_rng(seed)
    pick = []
    for kind in SERVE_KINDS:
        ok = [i for i, q in enumerate(qs) if serve_kind(q) == kind and
              (q.system.n <= 250 ** 3 if kind != "csr" else q.system.n <= 500_000)]
        pick += [int(i) for i in rng.choice(ok, size=min(per_kind, len(ok)), replace=False)]
    return sorted(pick)


def serve_bench(args, dev: int):
    """The serving stream: a seeded mix of queries (2D heat n = 1e4..4e6, 3D heat
    n = 1e6..6.4e7, random CSR n = 1e5..2e6 with 1..32 generators; horizons
    100..2000 steps, m 20..60).  The CSR (Arnoldi) queries use FP32 storage;
    the heat (Lanczos) queries are served in FP64, because FP32 storage under
    the three-term recurrence floors near 1e-6 on their outputs (measured in
    this leg on the sampled heat queries: `heat_fp32_storage_err`).  A burst
    of all queries through the continuous-batching server measures capacity;
    then Poisson arrivals at 0.5 and 0.8 x capacity give queries/s and the
    p50 / p99 latency from kv_submit to the results on the host (at 0.8 x also
    per query kind).  The same mix run one query at a time without the server
    gives the served form's speed-up: in FP64 (the plain method), in the
    served precisions (the batching alone) and all in FP32.  The served bounds
    are compared with the FP64 GPU path on a random sample; the sampled served
    results are kept for the CPU leg, which compares them with the oracle."""
    import torch
    import paper_1804_01583_gb300 as kv

    def bound_error(got, ref):  # per output row, scaled by the row's largest |bound|
        worst = 0.0
        for r in range(ref["hi"].shape[0]):
            S = max(np.max(np.abs(ref["lo"][r])), np.max(np.abs(ref["hi"][r])))
            d = max(np.max(np.abs(got["lo"][r] - ref["lo"][r])), np.max(np.abs(got["hi"][r] - ref["hi"][r])))
            worst = max(worst, d / S if S > 0 else d)
        return worst

    qs = W.serving_mix(args.serve_queries, seed=0)
    ctx = kv.Context(args.serve_pool_gb << 30, device=dev)
    srv = kv.Server(ctx, slots=args.serve_slots)

    def drain(tickets, results, t_start):
        done = 0
        for t in list(tickets):
            r = srv.poll(t)
            if r is not None:
                results[tickets.pop(t)] = r
                done += 1
        return done

    # capacity: everything at once
    t0 = time.perf_counter()
    pend = {srv.submit(q): k for k, q in enumerate(qs)}
    burst = {}
    while pend:
        drain(pend, burst, t0)
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    cap = len(qs) / makespan
    # Poisson arrivals at 0.5 and 0.8 x capacity (the second is the headline)
    def poisson(load):
        rate = load * cap
        rng = np.random.default_rng(12345)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(qs)))
        pend, res = {}, {}
        t0 = time.perf_counter()
        k = 0
        while k < len(qs) or pend:
            now = time.perf_counter() - t0
            while k < len(qs) and arrivals[k] <= now:
                pend[srv.submit(qs[k])] = k
                k += 1
            drain(pend, res, t0)
            time.sleep(0.0002)
        return rate, res, time.perf_counter() - t0

    rate_half, res_half, el_half = poisson(0.5)
    lat_half = np.array([res_half[i]["latency_ms"] for i in range(len(qs))])
    rate, res, elapsed = poisson(0.8)
    st = srv.stats()
    srv.close()
    lat = np.array([res[i]["latency_ms"] for i in range(len(qs))])
    kinds = [serve_kind(q) for q in qs]
    per_kind = {}
    for kind in SERVE_KINDS:
        lk = np.array([lat[i] for i in range(len(qs)) if kinds[i] == kind])
        per_kind[kind] = {"queries": int(lk.size), "p50_ms": float(np.percentile(lk, 50)),
                          "p99_ms": float(np.percentile(lk, 99)), "max_ms": float(np.max(lk))}
    # the same mix one query at a time through kv_run (no server): the plain
    # FP64 method, the served precisions, everything in FP32 storage
    sample = np.random.default_rng(7).choice(len(qs), size=min(24, len(qs)), replace=False)
    keep = set(int(i) for i in sample)
    plain, kept = {}, {}
    for prec in ("fp64", "served", "fp32"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k, q in enumerate(qs):
            qq = q if prec == "served" else W.Problem(**{**q.__dict__, "precision": prec})
            r = kv.solve(qq, ctx, expm_mode="propagate")
            if k in keep and prec != "served":
                kept[(prec, k)] = r
        plain[prec] = time.perf_counter() - t0
    # accuracy of the served results against the FP64 form on the same GPU,
    # and what FP32 storage would have given the sampled heat queries
    err_gpu64 = max(bound_error(res[k], kept[("fp64", k)]) for k in keep)
    heat32 = [bound_error(kept[("fp32", k)], kept[("fp64", k)]) for k in keep if serve_kind(qs[k]) != "csr"]
    ctx.close()
    osample = serve_oracle_sample(qs)
    SERVED_FOR_ORACLE.clear()
    SERVED_FOR_ORACLE.extend((i, qs[i], res[i]) for i in osample)
    return {"queries": len(qs), "mix": {kk: kinds.count(kk) for kk in SERVE_KINDS}, "slots": args.serve_slots,
            "pool_gb": args.serve_pool_gb, "capacity_qps": cap, "arrival_rate_qps": rate,
            "queries_per_s": len(qs) / elapsed,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "per_kind": per_kind,
            "at_half_capacity": {"arrival_rate_qps": rate_half, "queries_per_s": len(qs) / el_half,
                                 "p50_ms": float(np.percentile(lat_half, 50)),
                                 "p99_ms": float(np.percentile(lat_half, 99))},
            "max_running": st["max_running"], "memory_waits": st["memory_waits"],
            "csr_systems": {"built": st["systems_built"], "reused": st["systems_reused"],
                            "released_early": st["systems_released"]},
            "plain_fp64_sequential_s": plain["fp64"], "plain_served_precisions_sequential_s": plain["served"],
            "plain_fp32_sequential_s": plain["fp32"],
            "served_makespan_s": makespan,
            "speedup_over_plain_fp64": plain["fp64"] / makespan,
            "speedup_over_plain_same_precisions": plain["served"] / makespan,
            "speedup_over_plain_fp32": plain["fp32"] / makespan,
            "max_rel_bound_err_vs_fp64_gpu": err_gpu64, "fp64_gpu_sample": f"{len(sample)} random queries",
            "heat_fp32_storage_err": {"max": max(heat32) if heat32 else None, "queries": len(heat32),
                                      "note": "the sampled heat queries forced to FP32 storage, against FP64"},
            "oracle_sample": osample,
            "precision": "CSR queries fp32 storage / fp64 accumulation; heat queries fp64"}


# served results (index, query, result) that the CPU leg compares with the oracle
SERVED_FOR_ORACLE: list = []


def serve_oracle_errors() -> dict:
    """CPU leg: the sampled served results against the FP64 oracle
    (scale-normalised bound error per output row, as the parity tests)."""
    import oracle
    worst, per = 0.0, {}
    t0 = time.perf_counter()
    for i, q, got in SERVED_FOR_ORACLE:
        ref = oracle.run(W.Problem(**{**q.__dict__, "precision": "fp64"}))
        e = 0.0
        for r in range(ref["hi"].shape[0]):
            S = max(np.max(np.abs(ref["lo"][r])), np.max(np.abs(ref["hi"][r])))
            d = max(np.max(np.abs(got["lo"][r] - ref["lo"][r])), np.max(np.abs(got["hi"][r] - ref["hi"][r])))
            e = max(e, d / S if S > 0 else d)
        kind = serve_kind(q)
        per[kind] = max(per.get(kind, 0.0), e)
        worst = max(worst, e)
    return {"max_rel_bound_err_vs_fp64_oracle": worst, "per_kind": per, "queries": len(SERVED_FOR_ORACLE),
            "oracle_s": time.perf_counter() - t0}


def error_control_bench(dev: int):
    """Alg. 4 with the Lemma-1 error control on the 3D heat grid of 100^3
    (target 1e-6, Krylov dimension up to 600; the shape of the error-bound
    experiment of Sec. 5.3): the dimension the control picks, the bound, the
    time per query and the cost of the checkpoints."""
    import torch
    import paper_1804_01583_gb300 as kv
    out = {}
    ctx = kv.Context(4 << 30, device=dev)
    try:
        for label, prec in (("fp64", "fp64"), ("fp32", "fp32")):
            p = W.heat3d_100(m=600, steps=1000, precision=prec)
            cell = W.grid_index((100, 100, 100), (12, 12, 12))
            p.C_row_ptr, p.C_col, p.C_val = np.array([0, 1]), np.array([cell]), np.array([1.0])
            p.err_target = 1e-6
            sysh = kv.System(ctx, p.system, p.precision)
            ph = kv.ProblemHandle(ctx, sysh, p, expm_mode="propagate")
            ph.run(full=False)
            torch.cuda.synchronize()
            ctx.profile_enable(True)
            t0 = time.perf_counter()
            r = ph.run(full=True)
            ms = (time.perf_counter() - t0) * 1e3
            chk = sum(ctx.profile_read(nm)[1] for nm in ("error_expm", "error_bound"))
            kry = sum(ctx.profile_read(nm)[1] for nm in ("lanczos_fused", "lanczos_fused64", "stencil_alpha",
                                                         "stencil_update"))
            ctx.profile_enable(False)
            out[label] = {"m_used": int(r["m_used"][0]), "lemma1_bound": float(r["err_bound"][0]),
                          "ms_per_query": ms, "checkpoint_ms": chk, "krylov_ms": kry}
            ph.close()
            sysh.close()
    finally:
        ctx.close()
    out["workload"] = "heat3d-100^3, output cell (12,12,12), dt 0.02, 1000 steps, m <= 600, target 1e-6"
    return out


def configs_bench(dev: int) -> dict:
    """Configurations 1 and 2 as specified (20x20 2-D heat, m = 30, 500 steps;
    100^3 3-D heat, m = 40, 1000 steps; FP64 plain method) with the FP32
    storage form beside them: time per query (median of 5 after a warm-up,
    CUDA-synchronised wall time of kv_enqueue + kv_fetch), Krylov steps/s, and
    the first violation step (parity of both against the oracle is in the
    tests)."""
    import paper_1804_01583_gb300 as kv
    out = {}
    ctx = kv.Context(4 << 30, device=dev)
    try:
        for label, mk in (("2d-20x20", W.heat2d_20), ("3d-100^3", W.heat3d_100)):
            out[label] = {}
            for prec in ("fp64", "fp32"):
                p = mk(precision=prec)
                sysh = kv.System(ctx, p.system, p.precision)
                ph = kv.ProblemHandle(ctx, sysh, p)
                r = ph.run(full=False)
                ts = []
                for _ in range(5):
                    t0 = time.perf_counter()
                    ph.enqueue()
                    r = ph.fetch(full=False)
                    ts.append((time.perf_counter() - t0) * 1e3)
                ms = statistics.median(ts)
                out[label][prec] = {"ms_per_query": ms, "krylov_steps_per_s": p.m / (ms * 1e-3),
                                    "first_violation_step": int(r["viol_step"]), "m": p.m, "steps": p.steps,
                                    "n": int(p.system.n)}
                ph.close()
                sysh.close()
    finally:
        ctx.close()
    return out


def cpu_configs() -> dict:
    """The CPU oracle on the same two configurations (FP64, all host cores):
    wall time of one whole query (Krylov, exponentials, bounds)."""
    import oracle
    out = {}
    for label, mk in (("2d-20x20", W.heat2d_20), ("3d-100^3", W.heat3d_100)):
        p = mk()
        t0 = time.perf_counter()
        oracle.run(p, want_basis=False)
        out[label] = {"ms_per_query": (time.perf_counter() - t0) * 1e3, "cores": oracle.num_threads()}
    return out


def paper_heat_bench(dev: int, precisions=("fp64", "fp32"), forms=("grid", "csr", "grid1000"), pool_gb: int = 0):
    """The paper's own 3-D heat model (Sec. 5.3): the insulated cube with heat
    exchange at x = 1 (cell-centred reading), the heated region
    [0,0.4]x[0,0.2]x[0,0.1], the centre output, T = 20 by 0.02.
      * 100^3 with the Lemma-1 error control (target 1e-6, Krylov dimension up
        to 800), through the matrix-free grid path (FP64 and FP32 storage) and
        the CSR path (FP64): the dimension the control picks (the paper
        reports 544), the bound, the time per query and its Krylov and
        checkpoint parts;
      * 1000^3 (n = 1e9, the paper's largest run) through the grid path at a
        fixed Krylov dimension 30, FP64 and FP32: time per query and per
        iteration, and the Lemma-1 bound that dimension reaches (the paper's
        run needed k = 5932, beyond this library's Lanczos limit of 4096)."""
    import torch
    import paper_1804_01583_gb300 as kv
    out = {}
    kry_names = ("lanczos_fused64", "lanczos_fused", "stencil_alpha", "stencil_update", "stencil_init", "csr_spmv",
                 "csr_lanczos_update", "project")

    def timed(ctx, p, **kw):
        sysh = kv.System(ctx, p.system, p.precision)
        ph = kv.ProblemHandle(ctx, sysh, p, **kw)
        try:
            ph.run(full=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()  # the query as it runs (no events between the launches)
            r = ph.run(full=True)
            ms = (time.perf_counter() - t0) * 1e3
            ctx.profile_enable(True)  # then once more with every launch timed, for the parts
            ph.run(full=False)
            chk = sum(ctx.profile_read(nm)[1] for nm in ("error_expm", "error_bound"))
            kry = {nm: ctx.profile_read(nm) for nm in kry_names}
            ctx.profile_enable(False)
            kms = sum(v[1] for v in kry.values())
            launches = sum(v[0] for nm, v in kry.items() if nm.startswith(("lanczos", "stencil_update", "csr_spmv")))
            return {"m_used": int(r["m_used"][0]), "lemma1_bound": float(r["err_bound"][0]),
                    "ms_per_query": ms, "checkpoint_ms": chk, "krylov_ms": kms,
                    "krylov_ms_per_iteration": kms / max(1, launches),
                    "peak_centre_temperature": float(np.max(r["hi"][0])), "storage": ph.precision}
        finally:
            ph.close()
            sysh.close()

    ctx = kv.Context((pool_gb or 8) << 30, device=dev)
    try:
        if "grid" in forms:
            for prec in precisions:
                out[f"grid_100_{prec}"] = timed(ctx, W.paper_heat_grid(100, precision=prec, err_target=1e-6),
                                                expm_mode="propagate")
        if "csr" in forms:
            out["csr_100_fp64"] = timed(ctx, W.paper_heat(100, precision="fp64", err_target=1e-6),
                                        expm_mode="propagate")
    finally:
        ctx.close()
    if "grid1000" in forms:
        ctx = kv.Context(26 << 30, device=dev)
        try:
            for prec in precisions:
                out[f"grid_1000_{prec}"] = timed(ctx, W.paper_heat_grid(1000, precision=prec, m=30))
        finally:
            ctx.close()
    out["workload"] = ("paper heat3d (insulated, exchange 0.5 at x = 1), centre output, dt 0.02, 1000 steps; "
                       "100^3: m <= 800, target 1e-6 (paper: k = 544); 1000^3: m = 30 fixed")
    return out


def replicated_bench(dev: int, h: int = 20_000):
    """The replicated-block shape of Sec. 5.2 (n = 28 h, i = 8 h, o = 1, 300
    steps) at h = 20 000: one Krylov run of the transpose dynamics instead of
    8 h forward runs; time per query and where it goes."""
    import torch
    import paper_1804_01583_gb300 as kv
    out = {"workload": f"replicated 28x28 blocks h={h}: n={28 * h}, i={8 * h}, o=1, 300 steps, transposed"}
    t0 = time.perf_counter()
    p = W.replicated_blocks(h, simulate="transpose")
    out["host_build_s"] = time.perf_counter() - t0
    ctx = kv.Context(8 << 30, device=dev)
    try:
        t0 = time.perf_counter()
        sysh = kv.System(ctx, p.system, p.precision)
        ph = kv.ProblemHandle(ctx, sysh, p, expm_mode="propagate")
        out["problem_setup_s"] = time.perf_counter() - t0
        ph.run(full=False)
        torch.cuda.synchronize()
        ctx.profile_enable(True)
        k = 3
        t0 = time.perf_counter()
        for _ in range(k):
            r = ph.run(full=False)
        out["ms_per_query"] = (time.perf_counter() - t0) * 1e3 / k
        out["kernels_ms_per_query"] = {nm: ctx.profile_read(nm)[1] / k for nm in
                                       ("csr_spmv", "csr_spmm", "arnoldi_dots", "arnoldi_update", "project",
                                        "expm_propagate", "bounds") if ctx.profile_read(nm)[0]}
        ctx.profile_enable(False)
        out["krylov_runs"] = 1
        out["m_used"] = int(ph.fetch(full=True)["m_used"][0])
        out["first_violation_step"] = r["viol_step"]
        ph.close()
        sysh.close()
    finally:
        ctx.close()
    return out


def batched_bench(dev: int, nq: int = 64, reps: int = 5):
    """Small queries (the 20 x 20 heat configuration, FP64, m = 30, 500 steps):
    nq of them enqueued one after another on the context stream, against the
    same nq packed under one captured CUDA graph (kv_graph_*)."""
    import torch
    import paper_1804_01583_gb300 as kv
    qs = [W.heat2d_20() for _ in range(nq)]
    ctx = kv.Context(1 << 30, device=dev)
    systems = [kv.System(ctx, q.system, q.precision) for q in qs]
    handles = [kv.ProblemHandle(ctx, s, q) for s, q in zip(systems, qs)]
    g = kv.Graph(ctx, handles)

    def timed(fn):
        ts = []
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            for h in handles[-1:]:
                h.fetch(full=False)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(ts[1:])

    t_ind = timed(lambda: [h.enqueue() for h in handles])
    t_graph = timed(g.launch)
    same = all(np.array_equal(h.fetch(full=False)["hi"], handles[0].fetch(full=False)["hi"]) for h in handles)
    g.close()
    for h in handles:
        h.close()
    for s in systems:
        s.close()
    ctx.close()
    return {"workload": "heat2d-20x20 fp64 m=30 500 steps", "queries": nq, "ms_enqueued_one_by_one": t_ind,
            "ms_packed_graph": t_graph, "speedup": t_ind / t_graph, "queries_per_s_graph": nq / t_graph * 1e3,
            "results_identical": bool(same)}


def arnoldi_bytes(p) -> float:
    """Algorithmic bytes of the random-CSR Arnoldi run: per column and
    iteration j the SpMV (matrix values and column indices, one read of the
    input vector, one write), the dots pass (j+2 vectors) and the update pass
    (j+1 vectors read, w read and written)."""
    es = 8 if p.precision == "fp64" else 4
    s = p.system
    nnz = int(s.row_ptr[-1])
    N = s.n + (1 if s.b is not None else 0)
    tot = 0.0
    for _ in range(p.i):
        for j in range(p.m):
            tot += nnz * (4 + es) + 2 * N * es + (j + 2) * N * es + (j + 3) * N * es
    return tot


def polytope_leg(ph, p) -> dict:
    """The per-step LP of Sec. 2.1 on a finished query (kv_check_polytope):
    an unsafe triangle in the 2-D output plane (y1 >= a, y2 >= b,
    y1 + y2 <= c with a, b at 40% of the outputs' peak upper bounds) and a
    budget row on the 16 generators (sum z_j <= 4): one LP per step, i + 1 =
    18 rows, 38 constraints.  Host wall time of the call (uploads, the two
    launches, result copies)."""
    import torch
    r = ph.fetch(full=False)
    a, b = 0.4 * float(np.max(r["hi"][0])), 0.4 * float(np.max(r["hi"][1]))
    U = np.array([[-1.0, 0.0], [0.0, -1.0], [1.0, 1.0]])
    v = np.array([-a, -b, 3.0 * (abs(a) + abs(b))])
    Iz = np.zeros((1, p.i))
    Iz[0, :min(16, p.i)] = 1.0
    iota = np.array([4.0])
    ph.check_polytope(U, v, Iz, iota)  # warm-up
    reps, t = 3, []
    for _ in range(reps):
        t0 = time.perf_counter()
        res = ph.check_polytope(U, v, Iz, iota)
        t.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.median(t)
    S = p.steps + 1
    return {"ms_per_check": ms, "lps_per_s": S / (ms * 1e-3), "steps": S, "lp_rows": p.i + 1,
            "constraints": 3 + 1 + 2 * p.i, "first_violation_step": int(res["viol_step"]),
            "failed_steps": int(np.sum(res["status"] != 0)),
            "note": "host wall time of kv_check_polytope (uploads, 2 launches, result copies)"}


def csr_bench(args, dev: int, n: int = 2_000_000, legs=None):
    """The random-CSR workload (n = 2e6, 16 generators + the fixed column,
    m = 60, 2000 steps) in FP64 and FP32: time per query, Arnoldi GB/s; and
    the same query by the transpose dynamics (Sec. 4.1: 2 runs on A'^T from
    the output rows instead of 17 on A')."""
    import torch
    import paper_1804_01583_gb300 as kv
    out = {}
    for prec, sim in legs or (("fp64", "forward"), ("fp32", "forward"), ("fp64", "transpose"), ("fp32", "transpose")):
        p = W.random_csr_problem(n, seed=0, precision=prec)
        p.simulate = sim
        ctx = kv.Context((getattr(args, "pool_gb", 0) or 40) << 30, device=dev)
        sysh = kv.System(ctx, p.system, p.precision)
        ph = kv.ProblemHandle(ctx, sysh, p, expm_mode="propagate")
        ph.enqueue()
        ph.fetch(full=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()  # the query as it runs (no events between the launches)
        k = 2
        for _ in range(k):
            ph.enqueue()
        ph.fetch(full=False)
        ms = (time.perf_counter() - t0) * 1e3 / k
        ctx.profile_enable(True)  # then with every launch timed, for the per-kernel parts
        for _ in range(k):
            ph.enqueue()
        ph.fetch(full=False)
        kern = {}
        for name in ["csr_spmm", "csr_spmv", "row_dot", "arnoldi_dots", "arnoldi_update", "expm_propagate",
                     "init_norm", "scatter"]:
            nl, tms = ctx.profile_read(name)
            if nl:
                kern[name] = {"launches": nl // k, "ms_per_query": tms / k}
        lp = None
        if prec == "fp32" and sim == "forward":
            lp = polytope_leg(ph, p)
        ph.close()
        sysh.close()
        ctx.close()
        runs = p.o if sim == "transpose" else p.i
        key = prec if sim == "forward" else prec + "_transposed"
        out[key] = {"ms_per_query": ms, "runs": runs, "arnoldi_steps_per_s": runs * p.m / (ms * 1e-3),
                    "kernels": kern}
        if lp:
            out[key]["polytope"] = lp
        if sim == "forward":
            out[key]["arnoldi_GBps"] = arnoldi_bytes(p) / (ms * 1e-3) / 1e9
    if "fp64" in out and "fp32" in out:
        out["speedup_fp32_over_fp64"] = out["fp64"]["ms_per_query"] / out["fp32"]["ms_per_query"]
    if "fp32" in out and "fp32_transposed" in out:
        out["speedup_transposed_fp32"] = out["fp32"]["ms_per_query"] / out["fp32_transposed"]["ms_per_query"]
    out["workload"] = (f"random CSR n={n}, 10 off-diagonal nnz/row, i=17 (16 generators + fixed), o=2, m=60, "
                       f"2000 steps")
    return out


def kv_bytes_guess(p) -> int:
    # the FP64 single-pass form (three double vectors); the FP32 form (three
    # float vectors) runs on the same context after it
    return int(3 * 8 * p.system.n * 1.02) + (512 << 20)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kv", choices=["kv", "reference"])
    ap.add_argument("--workload", default="heat3d-1000", choices=["heat3d-1000", "heat3d-100", "heat2d-20", "heat3d-512"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--expm", default="per_step", choices=["per_step", "propagate"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=24)
    ap.add_argument("--no-compare-fp64", dest="compare_fp64", action="store_false")
    ap.add_argument("--no-serve", dest="serve", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-csr", dest="csr", action="store_false")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--csr-precision", default="fp32", choices=["fp32", "fp64"],
                    help="storage of the --csr-only query")
    ap.add_argument("--csr-only", type=int, default=0, metavar="N",
                    help="only the random-CSR query (forward, --csr-precision) at n = N (profiling case)")
    ap.add_argument("--paper-heat-form", default="grid,csr,grid1000",
                    help="forms of the paper-heat leg: grid (100^3), csr (100^3), grid1000 (1000^3)")
    ap.add_argument("--paper-heat-only", default="", choices=["", "fp64", "fp32"],
                    help="only the paper's heat experiment (100^3, target 1e-6) in one precision (profiling case)")
    ap.add_argument("--pool-gb", type=int, default=0,
                    help="device pool of the --csr-only and --paper-heat-only cases (GB; profiling runs keep it small)")
    ap.add_argument("--serve-queries", type=int, default=512)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-pool-gb", type=int, default=160)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.impl == "reference":
        if rank != 0:
            return
        p = workload(args.workload, "fp64")
        vals = []
        cb = None
        for _ in range(args.warmup + args.steps):
            cb = cpu_baseline(p, iters=args.cpu_iters)
            vals.append(cb["value"])
        v = statistics.median(vals[args.warmup:]) if args.steps else vals[-1]
        cb["value"] = v
        line = {"metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": 0, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": p.m * bytes_per_iteration(p) / v / 1e6,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": p.name, "n": p.system.n, "krylov_m": p.m, "precision": "fp64",
                           "sample": cb["sample"]},
                "cpu_baseline": cb,
                "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    if args.csr_only:
        import torch
        from paper_1804_01583_gb300 import build as kvbuild
        kvbuild.build()
        dev = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(dev)
        print(json.dumps({"metric": "random-CSR query ms", "csr_workload":
                          csr_bench(args, dev, n=args.csr_only, legs=((args.csr_precision, "forward"),))}))
        return
    if args.paper_heat_only:
        import torch
        from paper_1804_01583_gb300 import build as kvbuild
        kvbuild.build()
        dev = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(dev)
        print(json.dumps({"metric": "paper heat query ms",
                          "paper_heat": paper_heat_bench(dev, precisions=(args.paper_heat_only,),
                                                         forms=tuple(args.paper_heat_form.split(",")),
                                                         pool_gb=args.pool_gb)}))
        return
    if args.serve_only:
        import torch
        from paper_1804_01583_gb300 import build as kvbuild
        kvbuild.build()
        dev = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(dev)
        print(json.dumps({"metric": "serving queries/s", "serving": serve_bench(args, dev)}))
        return
    line, p = run_gpu(args, rank, world)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    if args.batched and world == 1:
        line["batched"] = batched_bench(dev)
        line["error_control"] = error_control_bench(dev)
        line["replicated"] = replicated_bench(dev)
        line["paper_heat"] = paper_heat_bench(dev)
        line["configs"] = configs_bench(dev)
    if args.csr and world == 1:
        line["csr_workload"] = csr_bench(args, dev)
    if args.serve and world == 1:
        line["serving"] = serve_bench(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(workload(args.workload, "fp64"), iters=args.cpu_iters)
        line["cpu_baseline"]["configs"] = cpu_configs()
        if "serving" in line and SERVED_FOR_ORACLE:
            oe = serve_oracle_errors()
            line["serving"]["max_rel_bound_err_vs_fp64_oracle"] = oe["max_rel_bound_err_vs_fp64_oracle"]
            line["serving"]["oracle_check"] = oe
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
