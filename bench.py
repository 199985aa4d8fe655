#!/usr/bin/env python
"""Benchmark of the random-walk hot path on one GB300 (or N, one process each).

Workload (one step): the synthetic random-walk benchmark on an R-MAT graph
(scale 20, edge factor 16, a = 0.57, b = c = 0.19, symmetrised, no self-loops
or duplicates): 2^24 walks of 64 steps from uniform start vertices, grouped
into bouquets by start vertex (bq_walk_batch, BOUQUET mode): the grouping
kernels plus the bouquet walk kernel with visit counting.  Inputs are resident
in HBM; L2 is flushed (256 MiB write) between timed steps.

Beside it, on the same line:
  naive         the one-walk-per-thread kernel on the same batch;
  aesc          AESC at eps = 0.1 (certified plan) on the tiny ER graph
                (n = 1000, m = 5000 plus a spanning path), all edges;
  e2e           the same walk batch through the C ABI with host buffers
                (starts in, visits out, copies inside the timed region);
  roofline      the bouquet walk kernel against the measured HBM copy peak,
                20 algorithmic bytes per walk step;
  cpu_baseline  the CPU oracle on a bounded sample of the same batch.

`--impl reference` times the CPU oracle instead (rank 0 only).
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

METRIC = ("walk-steps/s and AESC edges/s at ε (Bouquet vs naive GPU), % memory roofline; "
          "p50/p99 query latency")
N_WALKS = 1 << 24
N_STEPS = 64
BYTES_PER_STEP = 20  # 16-byte {row start, row end} + 4-byte neighbour id
WORKLOAD = "rmat20_ef16_walks2^24_len64"
CPU_SAMPLE_WALKS = 1 << 20
REF_SAMPLE_WALKS = 1 << 18
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["walks", "batched", "serving"], default="walks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-aesc", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mix", action="store_true",
                    help="leave out the short batched and serving legs of the default line")
    ap.add_argument("--mix-count", type=int, default=256,
                    help="batched workload: use the first N graphs of the 256-graph mix")
    ap.add_argument("--walk-lanes", type=int, default=None)
    ap.add_argument("--aggregate", type=int, default=None)
    ap.add_argument("--no-relabel", action="store_true",
                    help="walk the R-MAT graph without its degree-relabelled copy (hashed hub table)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seeds(rank: int):
    """(walk seed, start-vertex seed) of a rank's own batch: every rank walks
    a distinct batch of the same size (weak scaling, no data-path exchange)."""
    return 2024 + rank, 21 + rank


def max_over_ranks(dist, x: float, device) -> float:
    """The slowest rank's time (the job's time); x itself on one process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources each walk kernel (and the layout it reads) is built from
WALK_KERNEL_SOURCES = {
    "walk_hub_kernel": ("walks.cu", "internal.h", "hash.cuh", "edges.cuh"),
    "walk_relabel_kernel": ("walks.cu", "internal.h", "hash.cuh", "edges.cuh", "graph.cu"),
    "walk_relabel8_kernel": ("walks.cu", "internal.h", "hash.cuh", "edges.cuh", "graph.cu"),
}


def walk_kernel_digest(kernel: str = "walk_hub_kernel") -> str:
    """sha256 (16 hex digits) of the sources the walk kernel is built from."""
    h = hashlib.sha256()
    for name in WALK_KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2410_14056_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def walk_kernel_traffic(kernel: str = "walk_hub_kernel"):
    """dram bytes per launch from the committed ncu summary of `kernel`, if it
    was taken on the current kernel sources (else None)."""
    if kernel not in WALK_KERNEL_SOURCES:
        return None
    prof = os.path.join(ROOT, "profiles", f"{kernel}_rmat20.md")
    if not os.path.exists(prof):
        return None
    digest = walk_kernel_digest(kernel)
    vals = {}
    for line in open(prof):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != digest:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi samples (every 25 ms) while the timed region runs; entering
    waits (at most 3 s) for the first sample, so that a short timed region is
    still covered."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return self
        t_end = time.perf_counter() + 3.0
        while not self.lines and self.proc.poll() is None and time.perf_counter() < t_end:
            time.sleep(0.005)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(g, starts, seed):
    """The C oracle on the host cores, single-threaded and on every core.

    All-cores variant: one thread per core, each running the oracle's walk
    batch on its own contiguous slice of the starts (the oracle call releases
    the GIL).  Each slice numbers its walks from 0, so the walks differ from
    the GPU batch's, but the work (starts, steps, graph) is the same."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    sample = starts[:CPU_SAMPLE_WALKS]
    t0 = time.perf_counter()
    oracle.walk_batch(g, seed, sample, N_STEPS)
    dt1 = time.perf_counter() - t0
    single = {"value": sample.size * N_STEPS / dt1, "unit": "walk-steps/s", "cores": 1, "kind": "oracle",
              "sample": f"first {sample.size} walks of the batch x {N_STEPS} steps, "
                        f"single-threaded C oracle, {dt1:.1f} s"}
    cores = os.cpu_count() or 1
    big = starts[:min(starts.size, CPU_SAMPLE_WALKS * cores)]
    slices = np.array_split(big, cores)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as pool:
        list(pool.map(lambda sl: oracle.walk_batch(g, seed, sl, N_STEPS), slices))
    dtn = time.perf_counter() - t0
    return {"value": big.size * N_STEPS / dtn, "unit": "walk-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"first {big.size} walks of the batch x {N_STEPS} steps, C oracle on {cores} threads "
                      f"(one contiguous slice each, walk ids from 0 per slice), {dtn:.1f} s",
            "single_thread": single}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import concurrent.futures as cf

    import numpy as np

    import oracle
    from workloads import rmat20, uniform_starts
    g = rmat20()
    starts = uniform_starts(g, N_WALKS, 21)
    cores = os.cpu_count() or 1
    # one contiguous slice of the batch per host core (the oracle call
    # releases the GIL); each slice numbers its walks from 0
    sample = starts[:min(starts.size, REF_SAMPLE_WALKS * cores)]
    slices = np.array_split(sample, cores)
    with cf.ThreadPoolExecutor(cores) as pool:
        def step(parts):
            list(pool.map(lambda sl: oracle.walk_batch(g, 2024, sl, N_STEPS), parts))
        for _ in range(args.warmup):
            step([sl[:1024] for sl in slices])
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            step(slices)
            times.append(time.perf_counter() - t0)
    per_step = sum(times) / len(times)
    value = sample.size * N_STEPS / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "walk-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_walks_per_step": int(sample.size)},
        "cpu_baseline": {"value": value, "unit": "walk-steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample.size} walks of the batch x {N_STEPS} steps per step, "
                                   f"C oracle on {cores} threads (one contiguous slice each)"},
        "e2e": {"value": value, "unit": "walk-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aesc_measure(bq, torch, steps, warmup):
    """AESC at eps = 0.1 on the tiny ER graph, all edges, certified plan."""
    import numpy as np
    from workloads import er_with_path
    g = er_with_path(1000, 5000, 1)
    # spectrum of D^-1/2 A D^-1/2 (planner input, computed once on the host)
    A = np.zeros((g.n, g.n))
    for v in range(g.n):
        A[v, g.row(v).astype(np.int64)] = 1.0
    s = 1.0 / np.sqrt(g.degrees.astype(np.float64))
    lam = np.linalg.eigvalsh(A * s[:, None] * s[None, :])
    graph = bq.Graph.from_csr(g)
    graph.set_spectrum(float(lam[-2]), float(min(lam[0], 0.0)))
    tau, nw = bq.aesc_plan(graph, None, 0.1, 0.01)
    steps_per_call = float(np.sum(2.0 * tau.astype(np.float64) * nw))
    dtau = torch.from_numpy(tau.view(np.int32)).cuda()
    dnw = torch.from_numpy(nw.view(np.int32)).cuda()
    counts = torch.empty(4 * tau.size, dtype=torch.int32, device="cuda")
    sc = torch.empty(tau.size, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=counts, sc=sc)
    bq.sync()
    bq.profile_read()
    bq.profile_enable(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lat = []
    for _ in range(steps):
        ev0.record()
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=counts, sc=sc)
        ev1.record()
        ev1.synchronize()
        lat.append(ev0.elapsed_time(ev1))
    bq.sync()
    prof = bq.profile_read()
    bq.profile_enable(False)
    ms = sum(lat) / len(lat)
    kern_ms = prof["aesc_ms"] / max(prof["aesc_launches"], 1)
    naive = aesc_naive_row(bq, torch, graph, dtau, dnw, counts, ms, steps, warmup)
    # exact SC = effective resistance from the Laplacian's pseudoinverse (numpy, FP64)
    from workloads import all_edges
    uv = all_edges(g).astype(np.int64)
    lp = np.linalg.pinv(np.diag(A.sum(axis=1)) - A)
    exact = lp[uv[:, 0], uv[:, 0]] + lp[uv[:, 1], uv[:, 1]] - 2.0 * lp[uv[:, 0], uv[:, 1]]
    plain_err = float(np.max(np.abs(sc.cpu().numpy() - exact)))
    # the same certified plan with walks shared per vertex: every edge keeps at
    # least its N walks per side, so the same eps guarantee holds
    scounts = torch.empty_like(counts)
    ssc = torch.empty_like(sc)
    for _ in range(warmup):
        bq.aesc_estimate_shared(graph, 5, None, dtau, dnw, counts=scounts, sc=ssc)
    bq.sync()
    slat = []
    for _ in range(steps):
        ev0.record()
        bq.aesc_estimate_shared(graph, 5, None, dtau, dnw, counts=scounts, sc=ssc)
        ev1.record()
        ev1.synchronize()
        slat.append(ev0.elapsed_time(ev1))
    bq.sync()
    s_ms = sum(slat) / len(slat)
    nvert = np.zeros(g.n)
    tvert = np.zeros(g.n)
    for side in (0, 1):
        np.maximum.at(nvert, uv[:, side], nw.astype(np.float64))
        np.maximum.at(tvert, uv[:, side], tau.astype(np.float64))
    shared = {"ms_per_estimate": s_ms, "edges_per_s": tau.size / (s_ms / 1e3),
              "walk_steps_per_call": float(np.sum(nvert * tvert)),
              "max_abs_error_vs_exact": float(np.max(np.abs(ssc.cpu().numpy() - exact))),
              "speedup_vs_per_edge": ms / s_ms}
    return {
        "workload": f"G(n=1000, m=5000) seed 1 plus a spanning path (m={g.m}), all edges, eps=0.1, "
                    "delta=0.01, certified plan",
        "naive": naive,
        "shared_walks": shared,
        "max_abs_error_vs_exact": plain_err,
        "edges": int(tau.size), "edges_per_s": tau.size / (ms / 1e3),
        "walk_steps_per_call": steps_per_call,
        "walk_steps_per_s": steps_per_call / (ms / 1e3),
        "ms_per_estimate": ms, "p50_ms": statistics.median(lat),
        "p99_ms": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))],
        "count_kernel_ms": kern_ms,
        "count_kernel_gbs": steps_per_call * BYTES_PER_STEP / (kern_ms / 1e3) / 1e9,
    }


def aesc_naive_row(bq, torch, graph, dtau, dnw, counts, bouquet_ms, steps, warmup):
    """The same all-edges estimate with one walk per thread (BQ_AESC_NAIVE):
    Alg. 2 per walk against the bouquets of Alg. 3, at the same eps and plan.
    Its counters must equal the bouquet kernel's (checked here)."""
    ncounts = torch.empty_like(counts)
    nsc = torch.empty(dtau.numel(), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=ncounts, sc=nsc, naive=True)
    bq.sync()
    bq.profile_read()
    bq.profile_enable(True)
    lat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=ncounts, sc=nsc, naive=True)
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    bq.sync()
    prof = bq.profile_read()
    bq.profile_enable(False)
    # the timed bouquet estimate left its counters in `counts`
    if not torch.equal(ncounts, counts):
        raise RuntimeError("naive and bouquet AESC counters differ")
    ms = sum(lat) / len(lat)
    return {"ms_per_estimate": ms, "edges_per_s": dtau.numel() / (ms / 1e3),
            "count_kernel_ms": prof["aesc_ms"] / max(prof["aesc_launches"], 1),
            "bouquet_speedup": ms / bouquet_ms, "counters_equal_bouquet": True,
            "kernel": "aesc_naive_kernel: one walk per thread, plain CSR, per-walk atomics"}


POWERLAW_SCHEDULE = dict(tau_scale=2.0, tau_add=2, tau_max=64, n_scale=9.0, n_min=32)
PILOT_WALKS = 64  # pilot walks per side of the pilot plan
PILOT_Z = 3.0     # normal quantile of its half-width eps / 2


def aesc_cpu_baseline(g, seed, uv, tau, nw, n_edges=100_000):
    """The C oracle's AESC counters on a seeded sample of the edges, one
    contiguous slice per host core (the oracle call releases the GIL)."""
    import concurrent.futures as cf

    import numpy as np

    import oracle
    rng = np.random.default_rng(11)
    pick = np.sort(rng.choice(uv.shape[0], min(n_edges, uv.shape[0]), replace=False))
    cores = os.cpu_count() or 1
    parts = np.array_split(pick, cores)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(cores) as pool:
        list(pool.map(lambda p: oracle.aesc_counts(g, seed, uv[p], tau[p], nw[p]), parts))
    dt = time.perf_counter() - t0
    steps = float(np.sum(2.0 * tau[pick].astype(np.float64) * nw[pick]))
    return {"value": pick.size / dt, "unit": "edges/s", "cores": cores, "kind": "oracle",
            "sample": f"{pick.size} edges drawn uniformly (seed 11) with their plan, {steps:.3g} walk steps, "
                      f"C oracle counters on {cores} threads, {dt:.1f} s"}


def aesc_equal_accuracy(bq, torch, graph, tau, nw, ltau, lnw):
    """The AESC estimators compared at equal accuracy on all edges of the
    power-law graph.  Accuracy is the noise variance: the mean over edges of
    (est_seed_a - est_seed_b)^2 / 2 for two independent seeds, free of the
    truncation bias (the same Ŝ_tau for every variant) and of any reference.
    Each variant's walk counts are scaled by var_variant / var_plain (its
    variance per walk relative to the plain estimator's; variance falls as
    1/N), so all reach the plain estimator's variance; the table gives the
    time of one estimate at the scaled plan and the variance re-measured
    there."""
    import numpy as np
    k = tau.size

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()

    def run(kind, t_h, n_h, seed):
        dt, dn = dev(t_h), dev(n_h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        if kind == "plain" or kind == "pilot":
            _, sc = bq.aesc_estimate(graph, seed, None, dt, dn)
        elif kind == "push1":
            _, _, sc = bq.aesc_estimate_push(graph, seed, None, dt, dn, 1)
        elif kind == "push8":
            _, _, sc = bq.aesc_estimate_push(graph, seed, None, dt, dn, 8)
        else:
            _, _, sc = bq.aesc_estimate_shared(graph, seed, None, dt, dn)
        e1.record()
        e1.synchronize()
        bq.sync()
        return e0.elapsed_time(e1), sc.cpu().numpy()

    def measure(kind, t_h, n_h):
        run(kind, t_h, n_h, 105)  # warm-up
        ms, a = run(kind, t_h, n_h, 105)
        _, b = run(kind, t_h, n_h, 106)
        return ms, float(np.mean((a - b) ** 2) / 2.0)

    def scaled(n_h, t_h, factor):
        lim = (2**32 - 1) // (2 * t_h.astype(np.uint64) + 2)
        return np.minimum(np.maximum(np.ceil(n_h.astype(np.float64) * factor), 1), lim).astype(np.uint32)

    plans = {"plain": (tau, nw), "push1": (tau, nw), "push8": (tau, nw), "shared": (tau, nw), "pilot": (ltau, lnw)}
    base = {kind: measure(kind, *plan) for kind, plan in plans.items()}
    var0 = base["plain"][1]
    rows = {}
    for kind, (t_h, n_h) in plans.items():
        ms_b, var_b = base[kind]
        factor = var_b / var0
        walks_b = float(np.sum(n_h, dtype=np.float64))
        if kind == "plain":
            ms_s, var_s, n_s = ms_b, var_b, n_h
        else:
            n_s = scaled(n_h, t_h, factor)
            ms_s, var_s = measure(kind, t_h, n_s)
        rows[kind] = {"ms_at_plan": ms_b, "noise_var_at_plan": var_b, "n_scale": factor,
                      "ms_at_equal_accuracy": ms_s, "noise_var_at_equal_accuracy": var_s,
                      "edges_per_s_at_equal_accuracy": k / (ms_s / 1e3),
                      "walks_per_side_mean": float(np.sum(n_s, dtype=np.float64)) / k,
                      "walks_per_side_mean_at_plan": walks_b / k}
    best = min(rows, key=lambda r: rows[r]["ms_at_equal_accuracy"])
    return {"target_noise_var": var0, "variants": rows, "fastest_at_equal_accuracy": best,
            "note": "noise variance = mean over all edges of (est(seed 105) - est(seed 106))^2 / 2; "
                    "plain/push/shared use the scheduled plan, pilot its own plan; N scaled per variant"}


def aesc_powerlaw(bq, torch, steps, warmup, cpu=False):
    """AESC on the power-law graph (Chung-Lu n = 4M, mean degree 10,
    exponent 2.1, largest component), all edges at eps = 0.05 with the
    scheduled (uncertified) plan.  Accuracy checks: Foster residual
    |sum SC - (n-1)| / (n-1), and 1000 edges re-estimated with 16 x N and
    2 x tau."""
    import numpy as np
    from workloads import cached, chung_lu
    g = cached("chunglu4m_d10_g2.1_s3", lambda: chung_lu(4_000_000, 10, 2.1, seed=3))
    graph = bq.Graph.from_csr(g)
    eps = 0.05
    sched = bq.Schedule(POWERLAW_SCHEDULE["tau_scale"], POWERLAW_SCHEDULE["tau_add"],
                        POWERLAW_SCHEDULE["tau_max"], POWERLAW_SCHEDULE["n_scale"],
                        POWERLAW_SCHEDULE["n_min"], 0)
    tau, nw = bq.aesc_plan(graph, None, eps, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
    work = float(np.sum(2.0 * tau.astype(np.float64) * nw))
    dtau = torch.from_numpy(tau.view(np.int32)).cuda()
    dnw = torch.from_numpy(nw.view(np.int32)).cuda()
    counts = torch.empty(4 * tau.size, dtype=torch.int32, device="cuda")
    sc = torch.empty(tau.size, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=counts, sc=sc)
    bq.sync()
    bq.profile_read()
    bq.profile_enable(True)
    lat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate(graph, 5, None, dtau, dnw, counts=counts, sc=sc)
        e1.record()
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    bq.sync()
    prof = bq.profile_read()
    bq.profile_enable(False)
    ms = sum(lat) / len(lat)
    kern_ms = prof["aesc_ms"] / max(prof["aesc_launches"], 1)
    est = sc.cpu().numpy()
    naive = aesc_naive_row(bq, torch, graph, dtau, dnw, counts, ms, max(2, steps - 1), 1)
    foster = abs(float(est.sum()) - (g.n - 1)) / (g.n - 1)
    # re-estimate 1000 edges with 16 x N and 2 x tau (independent seed)
    rng = np.random.default_rng(7)
    pick = np.sort(rng.choice(tau.size, 1000, replace=False))
    from workloads import all_edges
    uv = all_edges(g)[pick]
    t2 = np.minimum(2 * tau[pick], 4096).astype(np.uint32)
    n2 = np.minimum(16 * nw[pick].astype(np.uint64), (2**32 - 1) // (2 * t2.astype(np.uint64) + 2)).astype(np.uint32)
    _, ref = bq.aesc_estimate_host(graph, 99, uv, t2, n2)
    diff = np.abs(est[pick] - ref)
    # the same estimate with the push phase (depth 1 where d(u) + d(v) < 2N)
    depth = torch.zeros(tau.size, dtype=torch.int32, device="cuda")
    acc = torch.zeros(4 * tau.size, dtype=torch.int64, device="cuda")
    bq.aesc_estimate_push(graph, 5, None, dtau, dnw, 1, depth=depth, acc=acc, sc=sc)
    bq.sync()
    plat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate_push(graph, 5, None, dtau, dnw, 1, depth=depth, acc=acc, sc=sc)
        e1.record()
        e1.synchronize()
        plat.append(e0.elapsed_time(e1))
    bq.sync()
    pms = sum(plat) / len(plat)
    pest = sc.cpu().numpy()
    dep = depth.cpu().numpy()
    pwork = float(np.sum(2.0 * (tau.astype(np.float64) - dep) * nw))
    pdiff = np.abs(pest[pick] - ref)
    # the same with pushes up to depth 8 (volume rule, support cap 512 from depth 2)
    bq.aesc_estimate_push(graph, 5, None, dtau, dnw, 8, depth=depth, acc=acc, sc=sc)
    bq.sync()
    dlat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate_push(graph, 5, None, dtau, dnw, 8, depth=depth, acc=acc, sc=sc)
        e1.record()
        e1.synchronize()
        dlat.append(e0.elapsed_time(e1))
    bq.sync()
    dest = sc.cpu().numpy()
    ddep = depth.cpu().numpy()
    ddiff = np.abs(dest[pick] - ref)
    deep = {"push_max": 8, "ms_per_estimate": sum(dlat) / len(dlat),
            "edges_per_s": tau.size / (sum(dlat) / len(dlat) / 1e3),
            "depth_histogram": np.bincount(ddep.astype(np.int64), minlength=9).tolist(),
            "walk_steps_per_call": float(np.sum(2.0 * (tau.astype(np.float64) - ddep) * nw)),
            "foster_residual": abs(float(dest.sum()) - (g.n - 1)) / (g.n - 1),
            "subset_1000_rms_diff_vs_16N_2tau": float(np.sqrt(np.mean(ddiff ** 2)))}
    push = {"edges_per_s": tau.size / (pms / 1e3), "ms_per_estimate": pms, "walk_steps_per_call": pwork,
            "frac_edges_depth1": float(dep.mean()),
            "foster_residual": abs(float(pest.sum()) - (g.n - 1)) / (g.n - 1),
            "subset_1000_max_abs_diff_vs_16N_2tau": float(pdiff.max()),
            "subset_1000_rms_diff_vs_16N_2tau": float(np.sqrt(np.mean(pdiff ** 2))),
            "plain_rms_diff_vs_16N_2tau": float(np.sqrt(np.mean(diff ** 2))), "deeper": deep}
    # the pilot plan: the same tau, N from PILOT_WALKS walks per side (z = PILOT_Z)
    t0 = time.perf_counter()
    ltau, lnw, _ = bq.aesc_plan_pilot(graph, 5, None, eps, sched, PILOT_WALKS, PILOT_Z, moments=False)
    plan_ms = (time.perf_counter() - t0) * 1e3
    ldtau = torch.from_numpy(ltau.view(np.int32)).cuda()
    ldnw = torch.from_numpy(lnw.view(np.int32)).cuda()
    bq.aesc_estimate(graph, 5, None, ldtau, ldnw, counts=counts, sc=sc)
    bq.sync()
    llat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate(graph, 5, None, ldtau, ldnw, counts=counts, sc=sc)
        e1.record()
        e1.synchronize()
        llat.append(e0.elapsed_time(e1))
    bq.sync()
    lms = sum(llat) / len(llat)
    lest = sc.cpu().numpy()
    ldiff = np.abs(lest[pick] - ref)
    pilot = {"n_pilot": PILOT_WALKS, "z": PILOT_Z, "plan_ms": plan_ms,
             "pilot_walk_steps": float(np.sum(2.0 * PILOT_WALKS * ltau.astype(np.float64))),
             "same_tau_as_schedule": bool(np.array_equal(ltau, tau)),
             "walk_steps_per_call": float(np.sum(2.0 * ltau.astype(np.float64) * lnw)),
             "nwalks_mean": float(lnw.mean()), "frac_edges_at_n_min": float(np.mean(lnw == sched.n_min)),
             "edges_per_s": tau.size / (lms / 1e3), "ms_per_estimate": lms,
             "foster_residual": abs(float(lest.sum()) - (g.n - 1)) / (g.n - 1),
             "subset_1000_max_abs_diff_vs_16N_2tau": float(ldiff.max()),
             "subset_1000_rms_diff_vs_16N_2tau": float(np.sqrt(np.mean(ldiff ** 2))),
             "subset_1000_frac_within_half_eps": float(np.mean(ldiff <= eps / 2))}
    # vertex-centric estimate: the walks of a vertex serve every edge at it
    # (N_x, tau_x = maxima over the edges at x), the same plan
    scounts = torch.empty(4 * tau.size, dtype=torch.int32, device="cuda")
    snused = torch.empty(2 * tau.size, dtype=torch.int32, device="cuda")
    bq.aesc_estimate_shared(graph, 5, None, dtau, dnw, counts=scounts, nused=snused, sc=sc)
    bq.sync()
    slat = []
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bq.aesc_estimate_shared(graph, 5, None, dtau, dnw, counts=scounts, nused=snused, sc=sc)
        e1.record()
        e1.synchronize()
        slat.append(e0.elapsed_time(e1))
    bq.sync()
    sms = sum(slat) / len(slat)
    sest = sc.cpu().numpy()
    uv_all = all_edges(g)
    vn = np.zeros(g.n, np.float64)
    vt = np.zeros(g.n, np.float64)
    for side in (0, 1):
        np.maximum.at(vn, uv_all[:, side], nw.astype(np.float64))
        np.maximum.at(vt, uv_all[:, side], tau.astype(np.float64))
    sdiff = np.abs(sest[pick] - ref)
    shared = {"edges_per_s": tau.size / (sms / 1e3), "ms_per_estimate": sms,
              "walk_steps_per_call": float(np.sum(vn * vt)),
              "foster_residual": abs(float(sest.sum()) - (g.n - 1)) / (g.n - 1),
              "subset_1000_max_abs_diff_vs_16N_2tau": float(sdiff.max()),
              "subset_1000_rms_diff_vs_16N_2tau": float(np.sqrt(np.mean(sdiff ** 2)))}
    equal = aesc_equal_accuracy(bq, torch, graph, tau, nw, ltau, lnw)
    graph.close()
    cpu_line = aesc_cpu_baseline(g, 5, uv_all, tau, nw) if cpu else None
    return {
        "naive": naive,
        "equal_accuracy": equal,
        "push_phase": push,
        "pilot_plan": pilot,
        "shared_walks": shared,
        "cpu_baseline": cpu_line,
        "workload": f"chung-lu n=4M d=10 gamma=2.1 LCC (n={g.n}, m={g.m}), all edges, eps={eps}, "
                    "scheduled plan (uncertified)",
        "schedule": POWERLAW_SCHEDULE,
        "edges": int(tau.size), "edges_per_s": tau.size / (ms / 1e3),
        "walk_steps_per_call": work, "walk_steps_per_s": work / (ms / 1e3),
        "ms_per_estimate": ms, "count_kernel_ms": kern_ms,
        "count_kernel_gbs": work * BYTES_PER_STEP / (kern_ms / 1e3) / 1e9,
        "tau_mean": float(tau.mean()), "nwalks_mean": float(nw.mean()),
        "foster_residual": foster,
        "subset_1000_max_abs_diff_vs_16N_2tau": float(diff.max()),
        "subset_1000_frac_within_eps": float(np.mean(diff <= eps)),
    }


def sampler_rows(bq, torch, graph, g, seed, st, args):
    """The bouquet walk batch with each sampler (independent, coupled with 8
    shared bits in groups of 32, the paper's SABA word taken literally), and
    how far walks from one start spread: 64 starts x 4096 walks x 16 steps,
    distinct vertices per start at steps 1, 4, 16 and distinct whole paths."""
    import numpy as np
    rows = {}
    rng = np.random.default_rng(5)
    live = np.flatnonzero(np.diff(g.offsets) > 0)
    picks = rng.choice(live, 64, replace=False).astype(np.uint32)
    dstarts = torch.from_numpy(np.repeat(picks, 4096).view(np.int32)).cuda()
    visits = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    for name, smp in (("independent", None), ("coupled_t8_w32", (1, 8, 32)), ("saba_literal", (2, 0, 1))):
        for _ in range(3):
            visits.zero_()
            bq.walk_batch(graph, seed, st, N_STEPS, sampler=smp, visits=visits)
        bq.sync()
        evs = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            visits.zero_()
            bq.walk_batch(graph, seed, st, N_STEPS, sampler=smp, visits=visits)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        bq.sync()
        ms = min(a.elapsed_time(b) for a, b in evs)
        paths = torch.zeros((dstarts.numel(), 17), dtype=torch.int32, device="cuda")
        bq.walk_batch(graph, seed + 1, dstarts, 16, sampler=smp, paths=paths)
        bq.sync()
        p = paths.cpu().numpy().reshape(64, 4096, 17)
        spread = {f"step{l}": float(np.mean([np.unique(p[i, :, l]).size for i in range(64)])) for l in (1, 4, 16)}
        whole = float(np.mean([np.unique(p[i], axis=0).shape[0] for i in range(64)]))
        rows[name] = {"ms_per_step": ms, "walk_steps_per_s": N_WALKS * N_STEPS / (ms / 1e3),
                      "distinct_vertices_per_start": spread, "distinct_paths_per_4096": whole}
    return rows


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    import paper_2410_14056_gb300 as bq
    from workloads import rmat20, uniform_starts

    if args.walk_lanes or args.aggregate is not None:
        t = bq.get_tuning()
        bq.set_tuning(walk_lanes=args.walk_lanes or t["walk_lanes"],
                      aggregate_visits=t["aggregate_visits"] if args.aggregate is None else args.aggregate)

    g = rmat20()
    seed, start_seed = rank_seeds(rank)
    starts = uniform_starts(g, N_WALKS, start_seed)
    # the walk graph gets the degree-relabelled copy (hubs found by id; measured
    # 8.81 against 8.96 ms per launch); the other graphs of the run do not
    relabel_before = bq.get_tuning()["hub_relabel"]
    bq.set_tuning(hub_relabel=0 if args.no_relabel else 1)
    graph = bq.Graph.from_csr(g)
    bq.set_tuning(hub_relabel=relabel_before)
    ginfo = graph.info()
    if not args.no_relabel and not ginfo["relabel_hubs"]:
        raise RuntimeError("the degree-relabelled copy of the walk graph was not built")
    st = torch.from_numpy(starts.view(np.int32)).cuda()
    visits = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def one_step(mode):
        visits.zero_()
        bq.walk_batch(graph, seed, st, N_STEPS, mode=mode, visits=visits)

    def timed(mode, steps, warmup):
        for _ in range(warmup):
            one_step(mode)
        bq.sync()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        bq.profile_read()
        bq.profile_enable(True)
        evs = []
        for k in range(steps):
            flush.fill_(k)  # evict the previous step's lines from L2 (untimed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            one_step(mode)
            e1.record()
            evs.append((e0, e1))
        torch.cuda.synchronize()
        bq.sync()
        if dist:
            dist.barrier()
        prof = bq.profile_read()
        bq.profile_enable(False)
        total_ms = max_over_ranks(dist, sum(a.elapsed_time(b) for a, b in evs), "cuda")
        return total_ms, prof

    autotune = None
    if args.walk_lanes is None:
        best_w, w_ms = bq.autotune_walks(graph, seed, st, N_STEPS, visits)
        autotune = {"walk_lanes": best_w, "ms_per_candidate_1_2_4": w_ms}
    with ClockSampler(local) as clocks:
        total_ms, prof = timed(bq.MODE_BOUQUET, args.steps, args.warmup)
    ms_per_step = total_ms / args.steps
    steps_per_batch = N_WALKS * N_STEPS
    # the walk kernel that ran, as the library counted its launches
    launched = {k: v for k, v in prof["walk_kernels"].items() if v}
    if len(launched) != 1 or sum(launched.values()) != args.steps:
        raise RuntimeError(f"expected one walk kernel launch per step, the library reports {launched}")
    walk_kernel = f"walk_{next(iter(launched))}_kernel"
    if not args.no_relabel and walk_kernel not in ("walk_relabel_kernel", "walk_relabel8_kernel"):
        raise RuntimeError(f"no kernel on the relabelled copy ran ({launched})")
    value = whole_job_rate(world, steps_per_batch, ms_per_step / 1e3)
    walk_ms = prof["walk_ms"] / max(prof["walk_launches"], 1)
    group_ms = prof["group_ms"] / max(prof["group_launches"], 1)
    launches = prof["kernel_launches"]

    bouquet_visits = visits.clone()  # the last timed batch
    # the same kernel on the walks in input order (no grouping by start)
    bq.set_tuning(group_walks=0)
    ug_steps = max(3, args.steps // 2)
    ug_total, ug_prof = timed(bq.MODE_BOUQUET, ug_steps, 1)
    bq.set_tuning(group_walks=1)
    if not torch.equal(visits, bouquet_visits):
        raise RuntimeError("grouped and ungrouped walk batches gave different visit counts")
    ungrouped = {"ms_per_step": ug_total / ug_steps,
                 "walk_kernel_ms": ug_prof["walk_ms"] / max(ug_prof["walk_launches"], 1),
                 "pairs_ms": ug_prof["group_ms"] / max(ug_prof["group_launches"], 1),
                 "note": "bq_tuning.group_walks = 0: the same walk kernel on the walks in input order; "
                         "the grouped step's walk kernel and grouping times are walk_kernel_ms_grouped and "
                         "grouping_ms_per_step"}
    ungrouped["walk_kernel_ms_grouped"] = walk_ms
    ungrouped["grouping_gain_in_walk_kernel"] = ungrouped["walk_kernel_ms"] / walk_ms
    naive_ms, _ = timed(bq.MODE_NAIVE, max(3, args.steps // 2), 1)
    naive_ms /= max(3, args.steps // 2)
    if not torch.equal(visits, bouquet_visits):
        raise RuntimeError("the naive and bouquet walk kernels gave different visit counts")
    if int(bouquet_visits.to(torch.int64).sum()) != N_WALKS * N_STEPS:
        raise RuntimeError("the visit counts do not sum to walks x steps")

    peak, peak_kind = measured_peaks()
    algo_bytes = BYTES_PER_STEP * steps_per_batch
    achieved = algo_bytes / (walk_ms / 1e3) / 1e9
    traffic = walk_kernel_traffic(walk_kernel)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": walk_kernel,
                "kernel_ms": walk_ms,
                "algorithmic_bytes_per_launch": algo_bytes,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)"
                if peak_kind == "measured" else "fallback 6.8 TB/s"}

    e2e = None
    if not args.no_e2e:
        host_starts = torch.from_numpy(starts.view(np.int32)).pin_memory().numpy().view(np.uint32)
        host_visits = torch.zeros(g.n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        for _ in range(2):
            bq.walk_batch_host(graph, seed, host_starts, N_STEPS, visits=host_visits)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            host_visits[:] = 0
            bq.walk_batch_host(graph, seed, host_starts, N_STEPS, visits=host_visits)
        e2e_s = max_over_ranks(dist, (time.perf_counter() - t0) / args.steps, "cuda")
        e2e = {"value": whole_job_rate(world, steps_per_batch, e2e_s), "unit": "walk-steps/s",
               "h2d_bytes_per_step": int(starts.nbytes + 4 * g.n),
               "d2h_bytes_per_step": int(4 * g.n), "ms_per_step": e2e_s * 1e3,
               "api": "bq_walk_batch with BQ_HOST_IO (pinned host buffers)"}

    samplers = sampler_rows(bq, torch, graph, g, seed, st, args) if rank == 0 and not args.no_aesc else None

    aesc = aesc_pl = batched = serving = None
    if not args.no_aesc and rank == 0:
        aesc = aesc_measure(bq, torch, max(5, args.steps), args.warmup)
        aesc_pl = aesc_powerlaw(bq, torch, 3, 1, cpu=not args.no_cpu_baseline)
    if not args.no_mix and rank == 0:
        graph.close()  # the walk graph is not needed by the mixed legs
        batched = batched_measure(bq, torch, SHORT_MIX_GRAPHS, 4, 1)
        serving = serving_measure(bq, torch, SHORT_SERVE_REQUESTS, SHORT_SERVE_SECONDS, 1,
                                  max_requests=SHORT_SERVE_MAX)

    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = cpu_baseline(g, starts, seed)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "walk-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "graph": g.describe(),
                       "n_walks_per_gpu": N_WALKS, "n_steps": N_STEPS,
                       "starts": "uniform over non-isolated vertices (seeded)",
                       "mode": "BOUQUET, independent sampler", "tuning": bq.get_tuning(),
                       "walk_kernel": walk_kernel,
                       "walk_kernel_source": "library launch counts (bq_profile.walk_kernel_launches)",
                       "walk_graph": {k: ginfo[k] for k in ("layout", "hub_slots", "packed_bits", "relabel_hubs",
                                                            "relabel_bits_id", "relabel_bits_off",
                                                            "relabel_bits_deg")},
                       "autotune": autotune,
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "parallelism": f"replicas x{world} (each GPU its own batch)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clocks.summary(),
            "grouping_ms_per_step": group_ms,
            "ungrouped": ungrouped,
            "naive": {"value": whole_job_rate(world, steps_per_batch, naive_ms / 1e3), "unit": "walk-steps/s",
                      "ms_per_step": naive_ms,
                      "bouquet_speedup": naive_ms / ms_per_step,
                      "visits_equal_bouquet": True},
            "samplers": samplers,
            "aesc": aesc,
            "aesc_powerlaw": aesc_pl,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    graph.close()
    if dist:
        dist.destroy_process_group()


def read_peaks(bq, torch):
    """Measured read ceilings through the library's probe: a 48 MiB buffer
    read 200 times in one launch (L2-resident once warm) and a 4 GiB buffer
    read twice (HBM).  GB/s of bytes read."""
    small = torch.ones(12 << 20, dtype=torch.int32, device="cuda")
    big = torch.ones(1 << 30, dtype=torch.int32, device="cuda")
    out = {"l2_read_gbs": bq.read_bandwidth(small, 200), "hbm_read_gbs": bq.read_bandwidth(big, 2),
           "how": "bq_profile_read_bandwidth: 48 MiB x 200 reads and 4 GiB x 2 reads, one launch each, "
                  "16-byte ld.global.cg loads, CUDA events"}
    del small, big
    torch.cuda.empty_cache()
    return out


def batched_measure(bq, torch, mix_count, steps, warmup, small_n=20_000):
    """Batched AESC over the first mix_count graphs of the 256-graph mix: all
    edges of every graph at its own eps (scheduled plan), one persistent
    launch replayed as a CUDA graph, against one bq_aesc_estimate per graph;
    the same comparison on the mix's small graphs alone (n <= small_n),
    where per-call launches and kernel tails, not walks, set the time."""
    import numpy as np
    from workloads import batched_mix

    mix = batched_mix(count=max(1, mix_count))
    sched = bq.Schedule(POWERLAW_SCHEDULE["tau_scale"], POWERLAW_SCHEDULE["tau_add"],
                        POWERLAW_SCHEDULE["tau_max"], POWERLAW_SCHEDULE["n_scale"],
                        POWERLAW_SCHEDULE["n_min"], 0)
    queries, host_plans, work = [], [], []
    for i, (g, eps) in enumerate(mix):
        graph = bq.Graph.from_csr(g)
        tau, nw = bq.aesc_plan(graph, None, eps, 0.01, mode=bq.PLAN_SCHEDULED, schedule=sched)
        work.append(float(np.sum(2.0 * tau.astype(np.float64) * nw)))
        queries.append({"graph": graph, "seed": 1000 + i, "uv": None,
                        "tau": torch.from_numpy(tau.view(np.int32)).cuda(),
                        "nwalks": torch.from_numpy(nw.view(np.int32)).cuda()})
        host_plans.append((tau, nw))
    steps_total = sum(work)
    edges = sum(int(q["tau"].numel()) for q in queries)
    best, tune_ms = bq.autotune_aesc(queries[::8])
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def compare(sel):
        """(sequential ms, batched ms, p50, p99, lat list) for the queries sel."""
        qs = [queries[i] for i in sel]
        batch = bq.Batch(qs)
        outs = batch.outputs

        def sequential():
            for q, (counts, sc) in zip(qs, outs):
                bq.aesc_estimate(q["graph"], q["seed"], None, q["tau"], q["nwalks"], counts=counts, sc=sc)
        for _ in range(max(1, warmup)):
            sequential()
        torch.cuda.synchronize()
        seq = []
        for k in range(steps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sequential()
            e1.record()
            e1.synchronize()
            seq.append(e0.elapsed_time(e1))
        bq.sync()
        ref = [c.clone() for c, _ in outs]
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            batch.run()
        torch.cuda.synchronize()
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg, stream=stream):
            batch.run()
        for _ in range(max(1, warmup)):
            cg.replay()
        torch.cuda.synchronize()
        lat = []
        for k in range(steps):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cg.replay()
            e1.record()
            e1.synchronize()
            lat.append(e0.elapsed_time(e1))
        bq.sync()
        if not all(torch.equal(r, c) for r, (c, _) in zip(ref, outs)):
            raise RuntimeError("batched counters differ from one call per graph")
        return batch, cg, sum(seq) / len(seq), sum(lat) / len(lat), lat

    batch, cg, seq_ms, ms, lat = compare(range(len(queries)))
    # kernel time of the counting launch (uncaptured run with event brackets)
    bq.profile_read()
    bq.profile_enable(True)
    batch.run()
    bq.sync()
    prof = bq.profile_read()
    bq.profile_enable(False)
    kern_ms = prof["aesc_ms"] / max(prof["aesc_launches"], 1)

    # end to end: plans in from pinned host memory, estimates out, per step
    pinned = [(torch.from_numpy(t.view(np.int32)).pin_memory(), torch.from_numpy(n.view(np.int32)).pin_memory())
              for t, n in host_plans]
    sc_host = [torch.empty(s.numel(), dtype=torch.float64).pin_memory() for _, s in batch.outputs]
    e2e_steps = max(1, steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for q, (ht, hn) in zip(queries, pinned):
            q["tau"].copy_(ht, non_blocking=True)
            q["nwalks"].copy_(hn, non_blocking=True)
        cg.replay()
        for (_, s), hs in zip(batch.outputs, sc_host):
            hs.copy_(s, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    batch.close()

    # the same queries with walks shared per vertex (bq_batch_create_shared)
    sbatch = bq.Batch(queries, shared=True)
    sstream = torch.cuda.Stream()
    with torch.cuda.stream(sstream):
        sbatch.run(sstream)
    torch.cuda.synchronize()
    scg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(scg, stream=sstream):
        sbatch.run(sstream)
    for _ in range(max(1, warmup)):
        scg.replay()
    torch.cuda.synchronize()
    slat = []
    for k in range(steps):
        flush.fill_(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        scg.replay()
        e1.record()
        e1.synchronize()
        slat.append(e0.elapsed_time(e1))
    bq.sync()
    q0 = queries[0]
    c1, _, _ = bq.aesc_estimate_shared(q0["graph"], q0["seed"], None, q0["tau"], q0["nwalks"])
    bq.sync()
    if not torch.equal(c1, sbatch.outputs[0][0]):
        raise RuntimeError("shared batch differs from a single vertex-centric call")
    s_ms = sum(slat) / len(slat)
    shared_row = {"ms_per_step": s_ms, "edges_per_s": edges / (s_ms / 1e3), "speedup_vs_plain_batch": ms / s_ms,
                  "note": "the vertex-centric estimator at the same plan (each edge gets at least its N walks "
                          "per side, so its variance is lower; see aesc_powerlaw.equal_accuracy)"}
    sbatch.close()
    del scg

    small = [i for i, (g, _) in enumerate(mix) if g.n <= small_n]
    by_size = None
    if small:
        sb, _, s_seq, s_ms, _ = compare(small)
        sb.close()
        by_size = {"graphs": len(small), "max_n": small_n,
                   "edges": sum(int(queries[i]["tau"].numel()) for i in small),
                   "walk_steps": sum(work[i] for i in small),
                   "sequential_ms": s_seq, "batched_ms": s_ms, "batching_speedup": s_seq / s_ms}

    peak, peak_kind = measured_peaks()
    probe = read_peaks(bq, torch)
    l2_peak = probe["l2_read_gbs"]
    achieved = steps_total * BYTES_PER_STEP / (kern_ms / 1e3) / 1e9
    for q in queries:
        q["graph"].close()
    return {
        "workload": f"first {len(mix)} graphs of the 256-graph batched mix (seed 4), all edges, "
                    "eps per graph from {0.05, 0.1, 0.2}, scheduled plan, one persistent launch replayed "
                    "as a CUDA graph",
        "graphs": len(mix), "vertices": sum(g.n for g, _ in mix), "edges": edges,
        "walk_steps_per_step": steps_total, "steps": steps,
        "edges_per_s": edges / (ms / 1e3), "walk_steps_per_s": steps_total / (ms / 1e3),
        "ms_per_step": ms, "p50_ms": statistics.median(lat),
        "p99_ms": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))],
        "sequential_one_call_per_graph_ms": seq_ms, "batching_speedup": seq_ms / ms,
        "small_graphs": by_size,
        "shared_walks": shared_row,
        "autotuned_aesc_lanes": best, "autotune_ms": tune_ms,
        "roofline": {"bound": "l2", "achieved": achieved, "unit": "GB/s", "kernel": "batch_count_kernel",
                     "kernel_ms": kern_ms, "peak_hbm": peak, "frac_hbm": achieved / peak,
                     "peak_l2_read_measured": l2_peak, "frac_l2": achieved / l2_peak,
                     "read_probe": probe,
                     "note": "algorithmic 20 B per walk step (all reads); the mix's graphs are L2-resident, "
                             "so the measured L2 read bandwidth is the ceiling"},
        "e2e": {"value": edges / e2e_s, "unit": "edges/s",
                "h2d_bytes_per_step": int(8 * edges), "d2h_bytes_per_step": int(8 * edges),
                "ms_per_step": e2e_s * 1e3},
        "gpu_launches_per_step": prof["kernel_launches"],
    }


def run_batched(args):
    """Batched AESC (256 graphs, one persistent launch captured in a CUDA
    graph): all edges of every graph at its own eps, scheduled plan."""
    import torch

    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq

    with ClockSampler(0) as clocks:
        r = batched_measure(bq, torch, args.mix_count, args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": r["edges_per_s"], "unit": "edges/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"batched_mix{r['graphs']}_aesc", "detail": r["workload"],
                   "graphs": r["graphs"], "vertices": r["vertices"], "edges": r["edges"],
                   "schedule": POWERLAW_SCHEDULE, "l2": "flushed between timed steps (256 MiB write, untimed)"},
        "roofline": r["roofline"], "e2e": r["e2e"], "batched": r,
        "gpu_launches_per_step": r["gpu_launches_per_step"], "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


# the short batched and serving legs of the default line
SHORT_MIX_GRAPHS = 48
SHORT_SERVE_REQUESTS = 1000
SHORT_SERVE_SECONDS = 1.5
SHORT_SERVE_MAX = 6000

SERVE_LOADS = (0.5, 0.8, 1.0)
SERVE_SATURATION_REQUESTS = 2000
SERVE_LOAD_SECONDS = 3.0
SERVE_SUBMITTERS = 12
SERVE_WAITERS = 128
# page-locked arena for request images: a 2000-request burst holds about 1 GB
SERVE_ARENA_BYTES = 2 << 30


def serving_graphs(bq, torch):
    """Eight resident graphs: two R-MAT scale 24 (edge factor 16), two
    4096 x 4096 grids with 5% of the edges deleted, four Chung-Lu graphs
    (n = 1M, mean degree 10, exponent 2.3, largest component)."""
    import numpy as np
    from workloads import cached, chung_lu
    from workloads import device as dev
    dgs = [dev.rmat(24, 16, seed=301), dev.rmat(24, 16, seed=302),
           dev.grid(4096, 4096, 0.05, 303), dev.grid(4096, 4096, 0.05, 304)]
    for s in (305, 306, 307, 308):
        h = cached(f"chunglu1m_d10_g2.3_s{s}", lambda s=s: chung_lu(1_000_000, 10.0, 2.3, s))
        dgs.append(dev.DeviceGraph(h.name, h.n, torch.from_numpy(np.asarray(h.offsets, np.int64)).cuda(),
                                   torch.from_numpy(np.asarray(h.nbrs, np.uint32).view(np.int32)).cuda()))
    torch.cuda.synchronize()
    graphs = [bq.Graph(d.n, d.offsets, d.nbrs, bq.DEVICE_PTRS | bq.BORROW) for d in dgs]
    return dgs, graphs


def serving_requests(dgs, count, rng, gen):
    """count requests: graph uniform over the eight, subset size log-uniform
    on [1, 1e5] with edges uniform over the graph's edges, eps ~ U[0.05, 0.2],
    a distinct seed each."""
    import numpy as np
    from workloads import device as dev
    out = []
    for _ in range(count):
        gi = int(rng.integers(len(dgs)))
        k = int(min(100_000, max(1, np.floor(np.exp(rng.uniform(0.0, np.log(100_001.0)))))))
        uv = dev.sample_edges(dgs[gi], k, gen)
        out.append((gi, uv, float(rng.uniform(0.05, 0.2)), int(rng.integers(0, 2**63))))
    return out


def serve_run(srv, reqs, arrivals, prompt=True):
    """Submit reqs at the given offsets (s) from a pool of submitting threads.
    prompt: wait for each request as soon as it is submitted, from a pool of
    waiting threads (a prompt client: a request's page-locked image returns to
    the server's pool when its results are read); else wait for all after the
    last submission (a burst: the waiting threads would slow the submitting
    ones).  Returns the latencies (arrival -> results ready on the host, ms)
    and the wall time from the first arrival to the last completion."""
    import concurrent.futures as cf
    lat = [0.0] * len(reqs)

    def submit(req, t_sched):
        t_start = time.perf_counter()
        rid = srv.submit(*req)
        return rid, (t_start - t_sched) * 1e3

    def wait(i, fut):
        rid, queued_ms = fut.result()
        _, _, server_ms = srv.wait(rid, timeout=600)
        lat[i] = queued_ms + server_ms

    with cf.ThreadPoolExecutor(SERVE_SUBMITTERS) as pool, cf.ThreadPoolExecutor(SERVE_WAITERS) as waiters:
        t0 = time.perf_counter()
        subs, done = [], []
        for i, (req, at) in enumerate(zip(reqs, arrivals)):
            t_sched = t0 + at
            # sleep to the arrival (no spinning: a spinning main thread holds
            # the GIL that the submitting threads need)
            dt = t_sched - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            f = pool.submit(submit, req, t_sched)
            if prompt:
                done.append(waiters.submit(wait, i, f))
            else:
                subs.append(f)
        for i, f in enumerate(subs):
            wait(i, f)
        for d in done:
            d.result()
        t_end = time.perf_counter()
    return lat, t_end - t0


def pct(v, q):
    s = sorted(v)
    return s[min(len(s) - 1, int(round(q * (len(s) - 1))))]


def serving_measure(bq, torch, sat_requests, load_seconds, warmup, max_requests=20000):
    """Serving: resident graphs, a burst of sat_requests requests at once
    (saturation), then Poisson arrivals at 0.5 / 0.8 / 1.0 of the measured
    saturation rate for load_seconds each; p50/p99 latency and edges/s."""
    import numpy as np

    dgs, graphs = serving_graphs(bq, torch)
    resident = sum(g.info()["device_bytes"] for g in graphs)
    rng = np.random.default_rng(909)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(910)
    cfg = bq.ServerConfig(device_budget_bytes=4 << 30, max_inflight=256, max_pending=65536,
                          pinned_arena_bytes=SERVE_ARENA_BYTES,
                          tasks_per_iteration=1 << 16, **POWERLAW_SCHEDULE)
    with bq.Server(graphs, cfg) as srv:
        # warm-up: a few requests through the whole path
        warm = serving_requests(dgs, max(3, warmup) * 4, rng, gen)
        serve_run(srv, warm, [0.0] * len(warm))
        # saturation: every request arrives at once
        sat_reqs = serving_requests(dgs, sat_requests, rng, gen)
        st0 = srv.stats()
        bq.profile_read()
        bq.profile_enable(True)
        lat, wall = serve_run(srv, sat_reqs, [0.0] * len(sat_reqs), prompt=False)
        prof = bq.profile_read()
        bq.profile_enable(False)
        st1 = srv.stats()
        sat_edges = sum(r[1].shape[0] for r in sat_reqs)
        sat_rps = len(sat_reqs) / wall
        steps = st1["walk_steps"] - st0["walk_steps"]
        kern_ms = prof["aesc_ms"]
        saturation = {"requests": len(sat_reqs), "edges": sat_edges, "wall_s": wall,
                      "requests_per_s": sat_rps, "edges_per_s": sat_edges / wall,
                      "walk_steps_per_s": steps / wall, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                      "iterations": st1["iterations"] - st0["iterations"],
                      "count_kernel_ms": kern_ms,
                      "worker_s": {k: st1[f"worker_{k}_s"] - st0[f"worker_{k}_s"]
                                   for k in ("admit", "launch", "complete", "idle")},
                      "planner_s": st1["planner_s"] - st0["planner_s"]}
        loads = []
        for f in SERVE_LOADS:
            rate = f * sat_rps
            count = int(min(max_requests, max(200, rate * load_seconds)))
            reqs = serving_requests(dgs, count, rng, gen)
            gaps = rng.exponential(1.0 / rate, count)
            arrivals = np.cumsum(gaps) - gaps[0]
            lat, wall = serve_run(srv, reqs, arrivals.tolist())
            edges = sum(r[1].shape[0] for r in reqs)
            loads.append({"offered": f, "rate_rps": rate, "requests": count, "edges": edges,
                          "edges_per_s": edges / wall, "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99),
                          "max_ms": max(lat)})
        final = srv.stats()
    peak, peak_kind = measured_peaks()
    achieved = steps * BYTES_PER_STEP / (kern_ms / 1e3) / 1e9 if kern_ms > 0 else None
    for g in graphs:
        g.close()
    return {
        "workload": "8 resident graphs (2 R-MAT scale 24 ef 16, 2 grids 4096^2 -5%, 4 Chung-Lu n=1M gamma 2.3), "
                    f"requests of log-uniform [1, 1e5] edges, eps ~ U[0.05, 0.2]: a {len(sat_reqs)}-request burst, "
                    f"then Poisson arrivals at 0.5 / 0.8 / 1.0 x the burst's rate for {load_seconds} s each",
        "graphs": [{"name": d.name, "n": d.n, "m": d.m} for d in dgs],
        "resident_graph_bytes": resident,
        "server": {"device_budget_bytes": cfg.device_budget_bytes, "max_inflight": cfg.max_inflight,
                   "tasks_per_iteration": cfg.tasks_per_iteration, "pinned_arena_bytes": cfg.pinned_arena_bytes,
                   "submitting_threads": SERVE_SUBMITTERS,
                   "waiting_threads": f"{SERVE_WAITERS} (Poisson loads wait for each request at once; the burst after its last submission)"},
        "saturation": saturation, "loads": loads,
        "p50_ms": {str(l["offered"]): l["p50_ms"] for l in loads},
        "p99_ms": {str(l["offered"]): l["p99_ms"] for l in loads},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak if achieved else None, "traffic": None,
                     "kernel": "serve_count_kernel", "kernel_ms": kern_ms, "peak_source": peak_kind},
        "e2e_note": "serving is end to end: pairs in from the host, estimates back to the host",
        "gpu_launches": prof["kernel_launches"], "server_stats": final,
    }


def run_serving(args):
    """Serving at the full request counts (2000-request burst, 3 s per load)."""
    import torch

    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_2410_14056_gb300 as bq

    with ClockSampler(0) as clocks:
        r = serving_measure(bq, torch, SERVE_SATURATION_REQUESTS, SERVE_LOAD_SECONDS, args.warmup)
    sat = r["saturation"]
    line = {
        "metric": METRIC, "value": sat["edges_per_s"], "unit": "edges/s", "n_gpus": 1,
        "steps": sat["requests"], "warmup": args.warmup, "ms_per_step": 1e3 * sat["wall_s"] / sat["requests"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "serving_8graphs_poisson", "detail": r["workload"], "graphs": r["graphs"],
                   "resident_graph_bytes": r["resident_graph_bytes"], "schedule": POWERLAW_SCHEDULE,
                   "server": r["server"], "step": "one request",
                   "l2": "inputs (resident graphs, 2 x 1.6 GB R-MAT) larger than L2"},
        "serving": r, "roofline": r["roofline"],
        "e2e": {"value": sat["edges_per_s"], "unit": "edges/s",
                "h2d_bytes_per_step": int(8 * sat["edges"] / sat["requests"]),
                "d2h_bytes_per_step": int(8 * sat["edges"] / sat["requests"]),
                "note": r["e2e_note"]},
        "gpu_launches": r["gpu_launches"], "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
