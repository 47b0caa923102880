#!/usr/bin/env python
"""Throughput benchmark of the GB300 LIETS QSGS generator.

One step = one full realization of the 400^3 workload (cd = 1e-4, spacing
s = 30, face/edge/corner G_ref = 0.01/0.0025/0.000625, solid fraction 0.80):
seeding, spacing, front construction, growth to the exact target.  The
metric is nodes/s = voxels generated per second of device time, summed over
ranks (each rank generates its own realizations: weak scaling, no
collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  ``--impl reference`` times the CPU oracle
on a bounded sample of the same workload (the comparison arm).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2602_11734_gb300 import workloads  # noqa: E402

METRIC = "nodes/s"
WORKLOAD = "single_400"
L2_FLUSH_BYTES = 256 << 20       # > 129 MB L2: written between timed steps
REF_SAMPLE_EDGE = 112            # --impl reference: per-step oracle sample
PEAK_PROBE_BLOCKS = 1 << 34      # Philox blocks timed by the Philox-only probe
# ALU peak of the growth kernel's work unit.  A Philox4x32-10 block is ten
# rounds of two 32x32->64 products, i.e. 40 32-bit multiply results (low and
# high halves), and an SM retires 64 32-bit integer multiplies per clock (the
# CUDA C++ Programming Guide's arithmetic-throughput table; 16 per clock in
# each of the 4 SM sub-partitions), so the ceiling is SMs x 64 x clock / 40
# blocks per second: 503.4 G blocks/s on 152 SMs at 2070 MHz.
INT_MULS_PER_SM_CLOCK = 64
PHILOX_BLOCK_MULS = 40
DEFAULT_SM_MHZ = 2070.0           # maximum SM clock of a GB300
# L2 probes: a 32 MiB buffer (resident in the 129 MB L2) read 64 times, and
# 2^30 scattered atomicOr reductions into the same buffer.
L2_PROBE_BYTES = 32 << 20
L2_PROBE_PASSES = 64
L2_PROBE_ATOMICS = 1 << 30
# Algorithmic bytes of one growth step (the per-step byte model of the
# method): read the front list (4 B per front voxel), gather its 3 x 3
# neighbour rows (36 B), one atomicOr per claim (4 B per claimed voxel),
# the prune test of the old front and the claimed voxels (36 B each) and
# the write of the next front (4 B per voxel of it).
BYTES_PER_FRONT_VOXEL = 4 + 36 + 36
BYTES_PER_CLAIM = 4 + 36
BYTES_PER_NEXT_FRONT_VOXEL = 4
CPU_BASELINE_TIMEOUT_S = 900


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help=">= 1")
    ap.add_argument("--no-batch", action="store_true", help="skip the 96-member batch report")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving report")
    ap.add_argument("--no-sweep", action="store_true", help="skip the 500^3 sweep report")
    ap.add_argument("--no-fullfield", action="store_true",
                    help="skip the full-field (Algorithm 2) comparator")
    ap.add_argument("--no-fontainebleau", action="store_true",
                    help="skip the Fontainebleau benchmark sweep (Sec. 3.3 setting)")
    ap.add_argument("--no-phases", action="store_true",
                    help="skip the three-phase label-map report")
    ap.add_argument("--no-sizes", action="store_true",
                    help="skip the 200^3..1000^3 size sweep in the paper's Fig. 3 setting")
    ap.add_argument("--no-tune", action="store_true",
                    help="library default launch shapes instead of the autotuner's")
    ap.add_argument("--edge", type=int, default=400,
                    help="grid edge of the timed workload (400 = the reported configuration; "
                         "smaller edges are for profiler captures)")
    ap.add_argument("--serve", action="store_true",
                    help="serving sweep only: 2000 requests, loads 0.25..1.2 of saturation")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_workload(rank: int, edge: int) -> dict:
    """The 400^3 parameters (at ``edge``^3) with this rank's own seed:
    ranks generate independent realizations (replicas, weak scaling)."""
    return dict(workloads.single_400(), seed=1 + rank, nx=edge, ny=edge, nz=edge)


def max_over_ranks(x: float, world: int, device) -> float:
    """The slowest rank's value (timing is max over ranks); no-op on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed / the max time."""
    return units_per_rank * world / (max_ms / 1000.0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs.

    Sampling starts before the region (``wait_first`` returns once the first
    sample is in, so nvidia-smi's start-up is not inside the region); each
    sample is stamped on arrival, and ``stop`` keeps the samples that arrived
    between ``begin`` and ``end``.  Only when the region is shorter than the
    sampling interval does it fall back to the samples around it."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 25

    def __init__(self, gpu_id: str):
        self.rows = []  # (arrival time, fields)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8:
                self.rows.append((time.perf_counter(), parts))

    def wait_first(self, timeout_s: float = 5.0) -> None:
        t0 = time.perf_counter()
        while (self.proc is not None and not self.rows and self.proc.poll() is None
               and time.perf_counter() - t0 < timeout_s):
            time.sleep(0.005)

    def stop(self, begin: float, end: float):
        if self.proc is None:
            return None
        time.sleep(2 * self.INTERVAL_MS / 1000.0)  # the sample in flight at `end`
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        return summarize_clocks(self.rows, begin, end)


def summarize_clocks(rows, begin: float, end: float):
    """Median SM clock, maximum clock and active throttle reasons of the
    samples stamped inside [begin, end]; with none inside, of the last
    sample before and the first after the region."""
    inside = [r for t, r in rows if begin <= t <= end]
    used = inside
    if not used:
        before = [r for t, r in rows if t < begin][-1:]
        after = [r for t, r in rows if t > end][:1]
        used = before + after
    sm = [float(r[0]) for r in used if r[0].replace(".", "").isdigit()]
    mx = [float(r[1]) for r in used if r[1].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in used for i in range(4) if r[4 + i].lower() == "active"})
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(sm), "samples_in_region": len(inside)}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def start_cpu_baseline(p: dict):
    """Times the CPU oracle on one full realization of ``p`` in a child
    process (one thread), started before the GPU work so that both run side
    by side; ``finish_cpu_baseline`` collects it."""
    code = ("import json, sys, time; sys.path.insert(0, %r)\n"
            "from oracle import oracle as O\n"
            "p = json.loads(%r); q = json.loads(%r)\n"
            "O.lib()\n"
            "ts = []\n"
            "for _ in range(3):\n"
            "    t0 = time.perf_counter(); O.run(q); ts.append(time.perf_counter() - t0)\n"
            "t0 = time.perf_counter(); r = O.run(p); dt = time.perf_counter() - t0\n"
            "print(json.dumps({'seconds': dt, 'solid': int(r.solid_count), "
            "'steps': int(r.steps), 'small_seconds': sorted(ts)[1]}))\n") % (
                ROOT, json.dumps(p), json.dumps(workloads.small_64()))
    return subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                            stderr=subprocess.PIPE, text=True), time.perf_counter()


def finish_cpu_baseline(handle, p: dict):
    proc, t_start = handle
    left = max(1.0, CPU_BASELINE_TIMEOUT_S - (time.perf_counter() - t_start))
    n = p["nx"] * p["ny"] * p["nz"]
    try:
        out, err = proc.communicate(timeout=left)
    except subprocess.TimeoutExpired:
        proc.kill()
        proc.communicate()
        return {"value": None, "unit": METRIC, "cores": 1, "host_cores": host_cores(),
                "kind": "oracle", "sample": f"one full {p['nx']}^3 realization: did not finish "
                                            f"within {CPU_BASELINE_TIMEOUT_S} s"}
    if proc.returncode != 0:
        return {"value": None, "unit": METRIC, "cores": 1, "host_cores": host_cores(),
                "kind": "oracle", "sample": "oracle failed: " + err.strip()[-200:]}
    r = json.loads(out.strip().splitlines()[-1])
    q = workloads.small_64()
    return {"value": n / r["seconds"], "unit": METRIC, "cores": 1, "host_cores": host_cores(),
            "kind": "oracle",
            "small_64": {"value": q["nx"] * q["ny"] * q["nz"] / r["small_seconds"],
                         "unit": METRIC, "seconds": r["small_seconds"],
                         "what": "the 64^3 workload (cd 0.002, s 0, solid 0.70), median of 3"},
            "sample": (f"one full realization of the timed workload itself ({p['nx']}^3, "
                       f"{r['seconds']:.1f} s, {r['steps']} steps; the single-threaded C "
                       f"oracle on one of the {host_cores()} host cores, run beside the GPU "
                       f"legs)")}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    p = dict(workloads.single_400(), nx=REF_SAMPLE_EDGE, ny=REF_SAMPLE_EDGE, nz=REF_SAMPLE_EDGE)
    O.lib()
    for _ in range(a.warmup):
        O.run(p)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        O.run(p)
        times.append(time.perf_counter() - t0)
    n = REF_SAMPLE_EDGE**3
    value = n * len(times) / sum(times)
    sample = (f"one full realization of the 400^3 parameters on a {REF_SAMPLE_EDGE}^3 box "
              "per step (single-threaded C oracle)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_edge": REF_SAMPLE_EDGE},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1,
                         "host_cores": host_cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))
    return 0


def tuned_single(Q, params: dict, enabled: bool) -> dict:
    """Autotuned growth shape for realizations like ``params`` (cached)."""
    if not enabled:
        return {"blocks": 0, "tile": 1, "cached": None}
    from paper_2602_11734_gb300 import tune
    return tune.tune_single(params)


def bench_sweep(Q, torch, dev, tune_on: bool) -> dict:
    """The 500^3 sweep: porosity {0.08..0.25} x spacing {10..50}, 25
    realizations, each single-instance.  Device time of seeding through the
    exact target per realization, L2 flushed before each."""
    from paper_2602_11734_gb300 import tune
    params = workloads.sweep_500()
    shape = tuned_single(Q, params[0], tune_on)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    g0 = Q.Generator(params[0], device=dev)
    tune.apply_single(g0, shape)
    g0.seed()
    g0.grow()  # warm-up (graph build)
    g0.close()
    times, voxels = [], 0
    for p in params:
        g = Q.Generator(p, device=dev)
        tune.apply_single(g, shape)
        s = g.stream
        with torch.cuda.stream(s):
            flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.seed()
        st = g.grow()
        e1.record(s)
        e1.synchronize()
        assert st.status == Q.QSGS_OK, st
        times.append(e0.elapsed_time(e1))
        voxels += p["nx"] * p["ny"] * p["nz"]
        g.close()
    return {"workload": "sweep_500", "realizations": len(params),
            "nodes_per_s": voxels / (sum(times) / 1000.0),
            "median_ms": statistics.median(times), "max_ms": max(times),
            "grow_shape": {k: shape[k] for k in ("blocks", "tile", "cached")}}


def bench_fullfield(Q, torch, dev, shape: dict) -> dict:
    """Comparator on the same 400^3 workload: the full-field sweep of
    Algorithm 2 (every voxel draws all seven growth blocks each step) against
    the list-driven step, same realization bit for bit.  Device time of
    seeding through the exact target, L2 flushed before each run."""
    from paper_2602_11734_gb300 import tune
    p = rank_workload(0, 400)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    out = {}
    for name, mode in (("lists", Q.QSGS_MODE_LIETS), ("fullfield", Q.QSGS_MODE_FULLFIELD)):
        g = Q.Generator(p, device=dev)
        tune.apply_single(g, shape)
        g.set_mode(mode)
        g.seed()
        g.grow()  # untimed: graph build
        s = g.stream
        with torch.cuda.stream(s):
            flush.fill_(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.seed()
        st = g.grow()
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": round(ms, 3), "nodes_per_s": 400**3 / (ms / 1000.0),
                     "philox_blocks": st.sum_draws, "solid": st.solid_count, "steps": st.steps}
        g.close()
    out["speedup_lists_over_fullfield"] = out["fullfield"]["ms"] / out["lists"]["ms"]
    out["same_realization"] = all(out["lists"][k] == out["fullfield"][k] for k in ("solid", "steps"))
    out["paper_context"] = ("RTX 4060: LIETS 24 s vs vectorized GPU QSGS 6 min at 400^3 "
                            "(Sec. 3.2), i.e. ~15x")
    return out


def bench_fontainebleau(Q, torch, dev) -> dict:
    """The Fontainebleau benchmark of Sec. 3.3, generation only: 500^3,
    porosity 0.15, S_d from a 225 um grain diameter and 4 um voxels,
    G_ref 8e-4 for every class, s = 0..40 step 5, five realizations per s.
    Device time of seeding through the exact target per realization."""
    runs, per_s = [], {}
    g0 = Q.Generator(workloads.fontainebleau(0, 0), device=dev)
    g0.seed()
    g0.grow()  # untimed warm-up
    g0.close()
    for sp in workloads.FONTAINEBLEAU_SPACINGS:
        for k in range(5):
            p = workloads.fontainebleau(sp, k)
            g = Q.Generator(p, device=dev)
            s = g.stream
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.seed()
            st = g.grow()
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            assert st.status == Q.QSGS_OK, st
            runs.append(ms)
            per_s.setdefault(sp, []).append((ms, st.n_seeds, st.steps))
            g.close()
    n = 500**3
    return {"workload": "fontainebleau_500", "realizations": len(runs),
            "nodes_per_s": n * len(runs) / (sum(runs) / 1000.0),
            "seed_probability": workloads.fontainebleau(0, 0)["cd"],
            "per_spacing": [{"s": sp, "median_ms": round(statistics.median(x[0] for x in v), 3),
                             "mean_seeds": statistics.mean(x[1] for x in v),
                             "mean_steps": statistics.mean(x[2] for x in v)}
                            for sp, v in sorted(per_s.items())]}


# Interactions of the interacting variant of the phases workload: phase 2
# enters phase 1 cells, phase 3 enters both (I per face / edge / corner).
PHASE_INTERACTIONS = [None, {1: (0.01, 0.0025, 0.000625)},
                      {1: (0.005, 0.0, 0.0), 2: (0.01, 0.0025, 0.0)}]


def bench_phases(Q, torch, dev) -> dict:
    """Three growing phases on the 400^3 box (Sec. 2.1 steps 4-5): volume
    fractions 0.45 / 0.20 / 0.10 of the domain, the rest matrix; each phase
    with the single-phase parameters otherwise.  Independent phases
    (reading R12), and the same phases interacting (R13,
    PHASE_INTERACTIONS).  Wall time of the whole label map (seeding, growth,
    label and blocked fetches of all three phases), after an untimed run."""
    base = workloads.single_400()
    phases = [dict(base, target_solid_fraction=f, seed=10 + k, spacing_s=s)
              for k, (f, s) in enumerate(((0.45, 30), (0.20, 15), (0.10, 0)))]

    def timed(interactions):
        Q.generate_phases(phases, device=dev, interactions=interactions)  # untimed warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        labels, stats = Q.generate_phases(phases, device=dev, interactions=interactions)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        counts = torch.bincount(labels.view(-1), minlength=4).cpu().tolist()
        return dt, counts, stats

    dt, counts, stats = timed(None)
    dti, counts_i, stats_i = timed(PHASE_INTERACTIONS)
    return {"workload": "phases_400", "phases": len(phases), "ms": round(dt * 1e3, 3),
            "nodes_per_s": 400**3 / dt,
            "label_counts": counts,
            "exact_targets": all(st.solid_count == st.target_count for st in stats),
            "interacting": {"ms": round(dti * 1e3, 3), "nodes_per_s": 400**3 / dti,
                            "label_counts": counts_i, "steps": [st.steps for st in stats_i],
                            "exact_targets": all(st.solid_count == st.target_count
                                                 for st in stats_i)}}


def bench_sizes(Q, torch, dev) -> dict:
    """The setting of the paper's throughput figure (Sec. 3.2, Fig. 3): cd
    2e-4, G_ref 8e-4 for every class, porosity 0.20, edges 200..1000, with
    diamond spacing s = 15 and without.  One realization per point, device
    time of seeding through the exact target after an untimed run of the
    same point, L2 flushed before it; library default launch shape."""
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    points = []
    for spacing in (True, False):
        for n in workloads.FIG3_EDGES:
            p = workloads.fig3_size(n, spacing)
            g = Q.Generator(p, device=dev)
            g.seed()
            g.grow()  # untimed: graph build
            s = g.stream
            with torch.cuda.stream(s):
                flush.fill_(2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            g.seed()
            st = g.grow()
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            points.append({"edge": n, "spacing_s": p["spacing_s"], "ms": round(ms, 3),
                           "nodes_per_s": n**3 / (ms / 1000.0), "steps": st.steps,
                           "exact_target": st.solid_count == st.target_count,
                           "workspace_mb": round(g.nbytes / 1e6, 1)})
            g.close()
    return {"workload": "fig3_sizes", "points": points,
            "paper_context": "RTX 4060, FP32: s = 15 peak 1.51e7 nodes/s at 600^3; "
                             "no spacing peak 2.70e7 nodes/s at 800^3 (Fig. 3)"}


def bench_batch(Q, torch, dev, tune_on: bool, repeats: int = 2) -> dict:
    """96 uneven realizations (edge 128..256, porosity U[0.10,0.30], spacing
    U{10..40}, cd 2e-4) advanced as one batch, against the same 96 run one
    after another on the single-realization path.  Device time of seeding
    through the exact target, L2 flushed before each timed run."""
    from paper_2602_11734_gb300 import tune
    params = workloads.batch_96()
    bshape = tune.tune_batch(params) if tune_on else {"blocks": 0, "tile": 1, "cached": None}
    gens = [Q.Generator(p, device=dev) for p in params]
    # The single path gets the autotuned shape of each member's size class.
    sshapes = {}
    for gen, p in zip(gens, params):
        key = Q.word_count(p).bit_length()
        if key not in sshapes:
            sshapes[key] = tuned_single(Q, p, tune_on)
        tune.apply_single(gen, sshapes[key])
    words = sum(Q.word_count(p) for p in params)
    batch = Q.Batch(len(params), words, device=dev)
    tune.apply_batch(batch, bshape)
    batch.set_members(gens)
    voxels = sum(p["nx"] * p["ny"] * p["nz"] for p in params)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = batch.stream

    def timed(fn, stream):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    batch.run()  # warm-up (builds the graph)
    batch_ms = min(timed(lambda: batch.run(), s) for _ in range(repeats))
    stats = batch.query()

    def run_single():
        for g in gens:
            g.seed()
            g.grow()
    run_single()
    # The single path runs each member on its own stream with a host wait per
    # realization; time it on the host around a device synchronisation.
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_single()
    torch.cuda.synchronize()
    single_ms = 1000 * (time.perf_counter() - t0)

    # The same members as single instances on concurrent streams: one host
    # thread per stream, each growing every SERVE_STREAMS-th member (every
    # generator has its own stream).
    import concurrent.futures as cf

    def worker(k):
        for i in range(k, len(gens), SERVE_STREAMS):
            gens[i].seed()
            gens[i].grow()

    with cf.ThreadPoolExecutor(SERVE_STREAMS) as ex:
        list(ex.map(worker, range(SERVE_STREAMS)))  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(SERVE_STREAMS) as ex:
        list(ex.map(worker, range(SERVE_STREAMS)))
    torch.cuda.synchronize()
    streams_ms = 1000 * (time.perf_counter() - t0)
    out = {"workload": "batch_96", "members": len(params), "voxels": voxels,
           "batch_ms": batch_ms, "realizations_per_s": len(params) / (batch_ms / 1000),
           "nodes_per_s": voxels / (batch_ms / 1000),
           "single_path_ms": single_ms,
           "single_path_realizations_per_s": len(params) / (single_ms / 1000),
           "speedup_vs_single_path": single_ms / batch_ms,
           "concurrent_streams_ms": streams_ms, "streams": SERVE_STREAMS,
           "concurrent_streams_realizations_per_s": len(params) / (streams_ms / 1000),
           "speedup_vs_concurrent_streams": streams_ms / batch_ms,
           "all_done": all(st.status == Q.QSGS_OK for st in stats),
           "grow_shape": {k: bshape.get(k) for k in ("blocks", "tile", "cached")}}
    batch.close()
    for g in gens:
        g.close()
    return out


SERVE_QUANTA = (2, 4, 8)           # growth steps per scheduling round
SERVE_LOADS = (0.75, 1.0)          # Poisson arrival rates, fractions of saturation
# The served configuration's full arrival-rate sweep, run at the default
# quantum (the last of SERVE_QUANTA); the other quanta take SERVE_LOADS.
SERVE_LOADS_SWEEP = (0.25, 0.5, 0.75, 0.9, 1.0, 1.2)
SERVE_STREAMS = 8                  # concurrent single instances of the stream arm


def bench_serve(torch, dev, n_requests: int, loads=SERVE_LOADS, quanta=SERVE_QUANTA,
                sweep=SERVE_LOADS_SWEEP) -> dict:
    """Continuous batching on the request mix (edge 64..512 with weights
    0.3/0.3/0.2/0.15/0.05, porosity U[0.08,0.30], spacing U{0..40}, cd 1e-4):
    per step quantum K, the closed-loop saturation rate (all requests at
    t = 0), then Poisson arrivals at fractions of it (`sweep` at the last,
    default quantum, `loads` at the others).  Latency =
    arrival to the uint8 phase map in pinned host memory.  Beside it, the
    same requests on the plain single-instance path, one after another, and
    as single instances on SERVE_STREAMS concurrent streams (host threads),
    every result copied to pinned host memory too."""
    import concurrent.futures as cf
    from paper_2602_11734_gb300 import qsgs as Q
    from paper_2602_11734_gb300 import serve as S
    params = workloads.serve_requests(n_requests)
    max_vox = max(p["nx"] * p["ny"] * p["nz"] for p in params)
    voxels = sum(p["nx"] * p["ny"] * p["nz"] for p in params)

    def run(arrivals, quantum):
        reqs = [S.Request(rid=i, params=p, arrival=float(t))
                for i, (p, t) in enumerate(zip(params, arrivals))]
        srv = S.Server(device=dev, max_members=256, step_quantum=quantum, keep_results=False,
                       staging_voxels=max_vox)
        t0 = time.perf_counter()
        srv.serve(reqs)
        wall = time.perf_counter() - t0
        out = S.summarize(reqs, wall_s=wall)
        out["rounds"] = srv.rounds
        srv.batch.close()
        return out

    run([0.0] * min(32, n_requests), quanta[-1])  # warm-up: graph build, allocator, pinning
    by_quantum = []
    for k in quanta:
        sat = run([0.0] * n_requests, k)
        points = []
        for f in (sweep if k == quanta[-1] else loads):
            rate = f * sat["requests_per_s"]
            pt = run(workloads.poisson_arrivals(n_requests, rate), k)
            pt.update({"load": f, "arrival_rate_per_s": rate})
            points.append(pt)
        by_quantum.append({"step_quantum": k, "saturation": sat, "sweep": points})

    def one(p, host):
        g = Q.Generator(p, device=dev)
        try:
            g.seed()
            g.grow()
            n = p["nx"] * p["ny"] * p["nz"]
            g.fetch(out=host[:n].view(g.shape))
        finally:
            g.close()

    staging = [torch.empty(max_vox, dtype=torch.uint8, pin_memory=True)
               for _ in range(SERVE_STREAMS)]
    for p in params[:16]:  # warm-up of the single path
        one(p, staging[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p in params:
        one(p, staging[0])
    single_s = time.perf_counter() - t0

    def worker(k):
        for i in range(k, len(params), SERVE_STREAMS):
            one(params[i], staging[k])

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(SERVE_STREAMS) as ex:
        list(ex.map(worker, range(SERVE_STREAMS)))
    streams_s = time.perf_counter() - t0
    best = max(by_quantum, key=lambda q: q["saturation"]["requests_per_s"])
    return {"workload": "serve_requests", "requests": n_requests,
            "latency": "arrival to the uint8 phase map in pinned host memory",
            "by_quantum": by_quantum,
            "single_path": {"requests_per_s": n_requests / single_s,
                            "nodes_per_s": voxels / single_s, "wall_s": single_s,
                            "what": "one request after another: seed, grow, u8 map to pinned "
                                    "host memory"},
            "concurrent_streams": {"streams": SERVE_STREAMS,
                                   "requests_per_s": n_requests / streams_s,
                                   "nodes_per_s": voxels / streams_s, "wall_s": streams_s,
                                   "what": "single instances on concurrent streams, one host "
                                           "thread each"},
            "saturation_vs_single_path": best["saturation"]["requests_per_s"] * single_s
                                         / n_requests,
            "saturation_vs_concurrent_streams": best["saturation"]["requests_per_s"] * streams_s
                                                / n_requests}


def main():
    a = parse()
    a.e2e_steps = max(1, a.e2e_steps)
    if a.impl == "reference":
        return run_reference(a)
    rank, world, local = dist_env()
    # The CPU baseline (rank 0, one GPU) starts first, as a child process:
    # the oracle's full realization of the timed workload runs on a host core
    # while the GPU legs run.
    cpu_handle = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline and not a.serve:
        cpu_handle = start_cpu_baseline(rank_workload(0, a.edge))
    import torch
    from paper_2602_11734_gb300 import build, qsgs as Q

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if a.serve:
        build.build()
        Q.load_library()
        res = bench_serve(torch, dev, 2000, quanta=(8,))
        if rank == 0:
            sat = res["by_quantum"][0]["saturation"]
            print(json.dumps({"metric": "requests/s", "value": sat["requests_per_s"],
                              "unit": "requests/s", "n_gpus": 1, "higher_is_better": True,
                              "data": "synthetic", "dtype": "u32",
                              "config": {"workload": "serve_requests"}, "served": res}),
                  flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    Q.load_library()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    from paper_2602_11734_gb300 import tune
    p = rank_workload(rank, a.edge)
    n_vox = p["nx"] * p["ny"] * p["nz"]
    shape = tuned_single(Q, p, not a.no_tune)  # before the timed region (cached per device)
    g = Q.Generator(p, device=dev)
    tune.apply_single(g, shape)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    s = g.stream

    for _ in range(max(3, a.warmup)):
        g.seed()
        st = g.grow()
    assert st.status == Q.QSGS_OK, st

    props = torch.cuda.get_device_properties(dev)
    gpu_id = f"GPU-{props.uuid}" if getattr(props, "uuid", None) else str(local)
    sampler = ClockSampler(gpu_id)
    sampler.wait_first()
    barrier()
    torch.cuda.synchronize()
    region_begin = time.perf_counter()
    times = []
    launches0 = g.query().launches
    launches_timed = 0
    for k in range(a.steps):
        with torch.cuda.stream(s):
            flush.fill_(k)  # evict L2 between timed steps (not timed)
        torch.cuda.synchronize()
        l0 = g.query().launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.seed()
        st = g.grow()
        e1.record(s)
        e1.synchronize()
        launches_timed += g.query().launches - l0
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop(region_begin, time.perf_counter())
    del launches0
    total_ms = max_over_ranks(sum(times), world, dev)
    value = job_rate(n_vox * a.steps, world, total_ms)

    # Kernel-level pass with the library's event profiler (not timed above).
    # k_grow is bound by integer ALU work: one Philox4x32-10 block per
    # front voxel and four targets of a direction class.  Its ceiling is the integer
    # multiply rate derived from the SM count and the sampled clock; the
    # rate the library's Philox-only probe reaches on this GPU is reported
    # beside it.  The L2 roof of the method's per-step byte model is set
    # against the L2 read bandwidth and atomic rate measured by the
    # library's own probes on this GPU, in this run.
    g.set_profiling(True)
    g.seed()
    st_prof = g.grow()
    prof = g.profile()
    g.set_profiling(False)
    grow_launches, grow_ms = prof["grow"]
    probe_out = torch.zeros(1, dtype=torch.int64, device=dev)
    probe_ms = min(Q.qsgs_bench_philox(PEAK_PROBE_BLOCKS, probe_out.data_ptr(), s.cuda_stream)
                   for _ in range(3))
    probe = PEAK_PROBE_BLOCKS / (probe_ms / 1000.0) / 1e9
    l2buf = torch.zeros(L2_PROBE_BYTES, dtype=torch.uint8, device=dev)
    l2_ms = min(Q.qsgs_bench_l2_read(l2buf.data_ptr(), L2_PROBE_BYTES, L2_PROBE_PASSES,
                                     probe_out.data_ptr(), s.cuda_stream) for _ in range(3))
    l2_gbs = L2_PROBE_BYTES * L2_PROBE_PASSES / (l2_ms / 1000.0) / 1e9
    red_ms = min(Q.qsgs_bench_l2_atomic(l2buf.data_ptr(), L2_PROBE_BYTES, L2_PROBE_ATOMICS,
                                        s.cuda_stream) for _ in range(3))
    red_gops = L2_PROBE_ATOMICS / (red_ms / 1000.0) / 1e9
    del l2buf
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clocks or {}).get("sm_mhz") or DEFAULT_SM_MHZ
    peak = sms * INT_MULS_PER_SM_CLOCK * sm_mhz * 1e6 / PHILOX_BLOCK_MULS / 1e9
    achieved = st_prof.sum_draws / (grow_ms / 1000.0) / 1e9
    pk, pk_kind = peaks()
    # The method's bytes of all growth steps of the realization: sum_front
    # is the sum of |A_t|, the claims are the voxels grown (solid - seeds),
    # and the next fronts sum to about the same as the fronts.
    claims = st_prof.solid_count - st_prof.n_seeds
    step_bytes = ((BYTES_PER_FRONT_VOXEL + BYTES_PER_NEXT_FRONT_VOXEL) * st_prof.sum_front
                  + BYTES_PER_CLAIM * claims)
    step_ms = sum(prof[k][1] for k in ("grow", "commit", "step_ctl"))
    l2_achieved = step_bytes / (step_ms / 1000.0) / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gblock/s",
                "frac": achieved / peak, "traffic": None, "kernel": "k_grow",
                "work": "Philox4x32-10 blocks drawn per second",
                "peak_kind": (f"derived: {sms} SMs x {INT_MULS_PER_SM_CLOCK} 32-bit integer "
                              f"multiplies per SM clock x {sm_mhz:.0f} MHz (sampled) / "
                              f"{PHILOX_BLOCK_MULS} multiplies per Philox4x32-10 block"),
                "probe": {"value": probe, "unit": "Gblock/s", "frac": achieved / probe,
                          "frac_of_peak": probe / peak,
                          "what": "qsgs_bench_philox: Philox4x32-10 alone on this GPU"},
                "draws": st_prof.sum_draws, "launches": grow_launches,
                "mean_launch_ms": grow_ms / max(1, grow_launches),
                "hbm_peak_gbs": pk["hbm_gbs"], "hbm_peak_kind": pk_kind,
                "l2": {"bound": "l2", "unit": "GB/s",
                       "algorithmic_bytes": step_bytes,
                       "bytes_model": (f"{BYTES_PER_FRONT_VOXEL + BYTES_PER_NEXT_FRONT_VOXEL} B "
                                       f"per front voxel-step + {BYTES_PER_CLAIM} B per claim"),
                       "step_ms": step_ms, "achieved": l2_achieved, "peak": l2_gbs,
                       "frac": l2_achieved / l2_gbs,
                       "frac_of_hbm": l2_achieved / pk["hbm_gbs"],
                       "peak_kind": (f"measured in this run: qsgs_bench_l2_read, "
                                     f"{L2_PROBE_BYTES >> 20} MiB x {L2_PROBE_PASSES} passes"),
                       "atomic_peak_gops": red_gops,
                       "claims_per_s": claims / (grow_ms / 1000.0) / 1e9,
                       "frac_atomic": claims / (grow_ms / 1000.0) / 1e9 / red_gops},
                "phases_ms": {k: round(v[1], 4) for k, v in prof.items()}}
    growth_ms = sum(prof[k][1] for k in ("grow", "commit", "step_ctl", "epilogue"))
    rates = {"growth_only_nodes_per_s": n_vox / (growth_ms / 1000.0),
             "front_voxel_updates_per_s": st_prof.sum_front / (grow_ms / 1000.0),
             "philox_blocks_per_s": st_prof.sum_draws / (grow_ms / 1000.0)}

    # End to end through the C ABI with host buffers: create, seed, grow and
    # copy the uint8 phase map to pinned host memory, every step.
    host = torch.empty(n_vox, dtype=torch.uint8, pin_memory=True)
    ws = torch.empty(g.nbytes, dtype=torch.uint8, device=dev)
    e2e_times = []
    for k in range(a.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = Q.qsgs_create(p, ws.data_ptr(), ws.numel(), s.cuda_stream)
        Q.qsgs_set_grow_blocks(h, shape["blocks"])
        Q.qsgs_set_grow_tile(h, shape["tile"])
        Q.qsgs_seed(h)
        rc, _ = Q.qsgs_grow_until(h, 0)
        Q.qsgs_fetch(h, host.data_ptr(), n_vox, Q.QSGS_FMT_U8, Q.QSGS_DST_HOST_MAPPED)
        Q.qsgs_destroy(h)
        t1 = time.perf_counter()
        if k:
            e2e_times.append(t1 - t0)
    e2e = {"value": n_vox * world / statistics.mean(e2e_times), "unit": METRIC,
           "h2d_bytes_per_step": ctypes.sizeof(Q.QsgsParams), "d2h_bytes_per_step": n_vox}

    cpu = None
    if cpu_handle is not None:
        cpu = finish_cpu_baseline(cpu_handle, p)
    batched = served = sweep = sizes = fullfield = fontainebleau = phases = None
    del g
    # The single-GPU reports below run at N = 1 only: under torchrun they
    # would hold every rank's GPU for minutes and repeat the same figures.
    if world > 1:
        a.no_phases = a.no_fontainebleau = a.no_fullfield = a.no_sweep = True
        a.no_sizes = a.no_batch = a.no_serve = True
    if not a.no_phases and a.edge == 400:
        phases = bench_phases(Q, torch, dev)
    if not a.no_fontainebleau and a.edge == 400:
        fontainebleau = bench_fontainebleau(Q, torch, dev)
    if not a.no_fullfield and a.edge == 400:
        fullfield = bench_fullfield(Q, torch, dev, shape)
    if not a.no_sweep and a.edge == 400:
        sweep = bench_sweep(Q, torch, dev, not a.no_tune)
    if not a.no_sizes and a.edge == 400:
        sizes = bench_sizes(Q, torch, dev)
    if not a.no_batch:
        batched = bench_batch(Q, torch, dev, not a.no_tune)
    if not a.no_serve:
        served = bench_serve(torch, dev, 2000)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": total_ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if a.edge == 400 else f"single_400 at {a.edge}^3",
                       "nx": a.edge, "ny": a.edge, "nz": a.edge, "cd": p["cd"],
                       "spacing_s": p["spacing_s"], "g_face": p["g_face"], "g_edge": p["g_edge"],
                       "g_corner": p["g_corner"], "solid_fraction": p["target_solid_fraction"],
                       "growth_steps": st.steps, "seeds": st.n_seeds,
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                       "grow_shape": {k: shape[k] for k in ("blocks", "tile", "cached")},
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "rates": rates, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_timed, "clocks": clocks, "sweep_500": sweep,
            "size_sweep": sizes, "fullfield_comparator": fullfield,
            "fontainebleau": fontainebleau, "phases": phases,
            "batched": batched, "served": served,
        }), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
