"""Write oracle results for the large workloads to tests/golden/*.jsonl.

Calls only the CPU oracle (``oracle/``) on parameter sets from
``paper_2602_11734_gb300.workloads``; nothing here touches the CUDA path.
Each line holds the parameters, the summary, the per-step front and claim
counts, and the SHA-256 of the final phase map as uint8[N] (x fastest).

    python tests/golden/make_golden.py small_64 single_400 sweep_500 batch_96 --jobs 6
    python tests/golden/make_golden.py serve_large --jobs 8
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2602_11734_gb300 import workloads  # noqa: E402

SETS = {
    "small_64": lambda: [workloads.small_64()],
    "single_400": lambda: [workloads.single_400()],
    "sweep_500": workloads.sweep_500,
    "batch_96": workloads.batch_96,
    "serve_small": lambda: [p for p in workloads.serve_requests() if p["nx"] <= 128][:40],
    # The large requests of the serving mix: the first three requests of
    # each of the edges 256, 400 and 512 among the 2000 (request ids 5, 7,
    # 15; 12, 20, 28; 14, 23, 34).
    "serve_large": lambda: [p for e in (256, 400, 512)
                            for p in [q for q in workloads.serve_requests() if q["nx"] == e][:3]],
}


def _one(args):
    name, idx, p = args
    from oracle import oracle as O
    t0 = time.time()
    r = O.run(p)
    dt = time.time() - t0
    return dict(set=name, index=idx, params=p, target_count=r.target_count,
                solid_count=r.solid_count, steps=r.steps, status=r.status,
                front_size=r.front_size, n_candidates=r.n_candidates, n_accepted=r.n_accepted,
                sha256_u8=hashlib.sha256(r.phase.tobytes()).hexdigest(),
                front_per_step=[int(v) for v in r.log["front"]],
                claimed_per_step=[int(v) for v in r.log["claimed"]],
                oracle_seconds=round(dt, 3))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("sets", nargs="+", choices=sorted(SETS))
    ap.add_argument("--jobs", type=int, default=1)
    a = ap.parse_args()
    from oracle import oracle as O
    O.build()
    for name in a.sets:
        todo = [(name, i, p) for i, p in enumerate(SETS[name]())]
        out_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.jsonl")
        with mp.get_context("spawn").Pool(a.jobs) as pool:
            rows = sorted(pool.imap_unordered(_one, todo), key=lambda r: r["index"])
        with open(out_path + ".tmp", "w") as f:
            for r in rows:
                f.write(json.dumps(r, sort_keys=True) + "\n")
        os.replace(out_path + ".tmp", out_path)
        print(f"{name}: {len(rows)} rows -> {out_path}", flush=True)


if __name__ == "__main__":
    main()
