"""Command line: generate QSGS realizations on the GPU and write them to disk.

    python -m paper_2602_11734_gb300 --size 400 400 400 --solid-fraction 0.8 \\
        --cd 1e-4 --g 0.01 0.0025 0.000625 --spacing 30 --seed 1 --out grain.raw

Writes each realization's phase map (1 = solid) as uint8 with x fastest
(``.raw``, or ``.npy`` with its shape (nz, ny, nx)), or as the library's
packed bit grid (``--packed``: word (z * ny + y) * ceil(nx / 32) + x / 32,
bit x & 31).  ``--count k`` writes k realizations with seeds seed ..
seed + k - 1 (``{i}`` in --out is replaced by the realization number).
Prints one JSON line of statistics per realization.  Every step runs in the
CUDA library; there is no CPU path.
"""
from __future__ import annotations

import argparse
import json
import os
import sys


def parse(argv=None) -> argparse.Namespace:
    ap = argparse.ArgumentParser(prog="python -m paper_2602_11734_gb300",
                                 description="QSGS porous-media generation (LIETS growth)")
    ap.add_argument("--size", type=int, nargs=3, metavar=("NX", "NY", "NZ"), required=True)
    ap.add_argument("--solid-fraction", type=float, default=None,
                    help="target solid fraction (phi_s); or give --target-count")
    ap.add_argument("--target-count", type=int, default=0, help="exact number of solid voxels")
    ap.add_argument("--cd", type=float, required=True, help="seed (core) distribution probability")
    ap.add_argument("--g", type=float, nargs=3, metavar=("FACE", "EDGE", "CORNER"), required=True,
                    help="reference growth probabilities of the face / edge / corner directions")
    ap.add_argument("--spacing", type=int, default=0, help="minimum L1 seed spacing s (0: none)")
    ap.add_argument("--seed", type=int, default=1, help="RNG seed of the first realization")
    ap.add_argument("--count", type=int, default=1, help="realizations (seeds seed, seed + 1, ...)")
    ap.add_argument("--max-steps", type=int, default=0, help="growth step limit (0: none)")
    ap.add_argument("--periodic", action="store_true", help="periodic (torus) domain")
    ap.add_argument("--packed", action="store_true", help="write the packed bit grid")
    ap.add_argument("--out", required=True, help="output path (.raw or .npy); {i} = realization")
    ap.add_argument("--device", type=int, default=0, help="CUDA device index")
    a = ap.parse_args(argv)
    if (a.solid_fraction is None) == (a.target_count == 0):
        ap.error("give exactly one of --solid-fraction and --target-count")
    if a.count < 1:
        ap.error("--count must be >= 1")
    if a.count > 1 and "{i}" not in a.out:
        ap.error("--count > 1 needs {i} in --out")
    if a.packed and a.out.endswith(".npy"):
        ap.error("--packed writes raw words: use a .raw path")
    return a


def params_of(a: argparse.Namespace, k: int) -> dict:
    """The qsgs parameter dict of realization k."""
    nx, ny, nz = a.size
    return dict(nx=nx, ny=ny, nz=nz, cd=a.cd, g_face=a.g[0], g_edge=a.g[1], g_corner=a.g[2],
                spacing_s=a.spacing, target_solid_fraction=a.solid_fraction or 0.0,
                target_count=a.target_count, seed=a.seed + k, max_steps=a.max_steps,
                periodic=1 if a.periodic else 0)


def main(argv=None) -> int:
    a = parse(argv)
    import numpy as np
    import torch
    from . import build
    from . import qsgs as Q
    build.build()
    Q.load_library()
    dev = torch.device("cuda", a.device)
    torch.cuda.set_device(dev)
    nx, ny, nz = a.size
    host = None
    for k in range(a.count):
        g = Q.Generator(params_of(a, k), device=dev)
        try:
            g.seed()
            st = g.grow()
            if a.packed:
                out = g.fetch(fmt="packed").cpu().numpy()
            else:
                if host is None:
                    host = torch.empty((nz, ny, nx), dtype=torch.uint8, pin_memory=True)
                g.fetch(out=host)
                out = host.numpy()
        finally:
            g.close()
        path = a.out.replace("{i}", str(k))
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        if path.endswith(".npy"):
            np.save(path, out)
        else:
            out.tofile(path)
        print(json.dumps({"path": path, "seed": a.seed + k, "steps": st.steps,
                          "status": st.status, "solid_count": st.solid_count,
                          "target_count": st.target_count, "front_size": st.front_size}),
              flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
