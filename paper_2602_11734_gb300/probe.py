"""Profiling entry points of the generator (used by the ncu summaries).

    python -m paper_2602_11734_gb300.probe grow [--edge 400] [--start 30] [--steps 2]
        One realization of the 400^3 workload (at edge^3) grown to step
        `start` with direct launches, then `steps` more: a profiler
        capture of the growth kernel skips `start` launches and takes the
        next ones (e.g. ncu -k regex:k_grow -s 30 -c 2).
    python -m paper_2602_11734_gb300.probe steps [--workload single_400 | --fig3 N]
        Per growth step of one realization: the front, the solid count and
        the event-timed device time of the growth and commit kernels (the
        library's event profiler, one step per call), as one JSON line.
    python -m paper_2602_11734_gb300.probe batch [--start 20] [--steps 2]
        The 96-member batch workload seeded, then advanced `start` steps and
        `steps` more with direct launches (one batched growth launch per
        step): a profiler capture of the batched growth kernel skips `start`
        launches (e.g. ncu -k regex:k_grow_batch -s 20 -c 2).

Both run the CUDA library only; nothing here computes voxels.
"""
from __future__ import annotations

import argparse
import json

from . import qsgs as Q
from . import workloads as W


def grow(edge: int, start: int, steps: int) -> dict:
    p = dict(W.single_400(), nx=edge, ny=edge, nz=edge)
    g = Q.Generator(p)
    try:
        g.seed()
        g.set_profiling(True)  # direct launches: every growth step is one launch
        g.grow(start)
        st = g.grow(steps)
        return {"steps": st.steps, "front": st.front_size, "solid": st.solid_count}
    finally:
        g.close()


def batch(start: int, steps: int) -> dict:
    params = W.batch_96()
    gens = [Q.Generator(p) for p in params]
    b = Q.Batch(len(params), sum(Q.word_count(p) for p in params))
    try:
        b.set_members(gens)
        b.seed()
        b.set_profiling(True)  # direct launches: every batch step is one growth launch
        b.advance(start)
        b.advance(steps)
        st = b.query()
        return {"members": len(st), "steps": max(x.steps for x in st),
                "solid": sum(x.solid_count for x in st)}
    finally:
        b.close()
        for g in gens:
            g.close()


def steps(params: dict) -> dict:
    g = Q.Generator(params)
    try:
        g.seed()
        g.grow()  # warm-up (and kernel set-up)
        g.set_profiling(True)
        g.seed()
        rows, prev = [], {"commit": 0.0, "grow": 0.0}
        while True:
            st = g.grow(1)
            pr = g.profile()
            rows.append({"t": st.steps, "front": st.front_size, "solid": st.solid_count,
                         "commit_us": round(1000 * (pr["commit"][1] - prev["commit"]), 2),
                         "grow_us": round(1000 * (pr["grow"][1] - prev["grow"]), 2)})
            prev = {"commit": pr["commit"][1], "grow": pr["grow"][1]}
            if st.status != Q.QSGS_RUNNING:
                break
        return {"nwords": g.words, "steps": rows,
                "commit_ms": round(sum(r["commit_us"] for r in rows) / 1000, 4),
                "grow_ms": round(sum(r["grow_us"] for r in rows) / 1000, 4)}
    finally:
        g.close()


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=("grow", "steps", "batch"))
    ap.add_argument("--edge", type=int, default=400)
    ap.add_argument("--start", type=int, default=30)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--workload", default="single_400")
    ap.add_argument("--fig3", type=int, default=0, help="edge of the Fig. 3 setting (s = 15)")
    a = ap.parse_args()
    from . import build
    build.build()
    Q.load_library()
    if a.mode == "grow":
        out = grow(a.edge, a.start, a.steps)
    elif a.mode == "batch":
        out = batch(a.start, a.steps)
    else:
        params = W.fig3_size(a.fig3, True) if a.fig3 else getattr(W, a.workload)()
        out = dict(steps(params), workload=f"fig3_{a.fig3}" if a.fig3 else a.workload)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
