"""Autotuner for the launch shape of the growth kernels.

A shape is (thread blocks, front tile): the blocks of k_grow / k_grow_batch
and the number of 32-word chunks of the candidate list a warp takes per grab
from the kernel's chunk dispenser.  Results never depend on the shape, only
the time does.

Single realization: every candidate shape is timed with ``qsgs_time_grow``,
which replays the growth kernel on the live state of a running realization
and leaves the realization exactly as it was, at a few points of a
representative run; the shape with the least summed time wins.

Batches: every candidate shape runs a fixed subset of the batch's members
from seeding to the end; the fastest wins.

Results are cached in a JSON file (``QSGS_TUNE_CACHE``, default
``~/.cache/qsgs/tune.json``) keyed by device, library build and workload
class, so a process tunes once per kind of workload.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import qsgs as Q

TILES = (1, 2, 4, 8)
BLOCKS_PER_SM = (1, 2, 3)  # k_grow holds three blocks per SM: at most one wave


def candidate_shapes(num_sms: int, blocks_per_sm=BLOCKS_PER_SM, tiles=TILES) -> list[tuple[int, int]]:
    """All (blocks, tile) pairs to time, one wave or less of blocks."""
    return [(b * num_sms, t) for b in blocks_per_sm for t in tiles]


def pick_best(timings: dict) -> tuple[int, int]:
    """The shape with the least summed time; ties go to the smaller grid,
    then the smaller tile (deterministic)."""
    return min(timings, key=lambda s: (sum(timings[s]), s[0], s[1]))


def _cache_path() -> str:
    return os.environ.get("QSGS_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "qsgs", "tune.json")


def _build_id() -> str:
    try:
        st = os.stat(Q.LIB_PATH)
        return f"{Q.qsgs_version()}-{st.st_size}-{int(st.st_mtime)}"
    except OSError:
        return str(Q.qsgs_version())


def _device_id(device) -> tuple[str, int]:
    import torch
    prop = torch.cuda.get_device_properties(device)
    return prop.name, prop.multi_processor_count


def cache_key(kind: str, device, words: int) -> str:
    name, sms = _device_id(device)
    bucket = int(math.log2(max(1, words)))  # workloads within a factor of two share a shape
    return f"{kind}|{name}|{sms}|{_build_id()}|w2^{bucket}"


def _load_cache() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value: dict) -> None:
    path = _cache_path()
    cache = _load_cache()
    cache[key] = value
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only costs a re-tune


def tune_single(params: dict, device=None, points=(0.3, 0.55, 0.8), reps: int = 5,
                use_cache: bool = True) -> dict:
    """Shape for single realizations like ``params``; returns
    {"blocks", "tile", "timings_ms", "cached"}."""
    import torch
    device = torch.device(device) if device is not None else torch.device(
        "cuda", torch.cuda.current_device())
    key = cache_key("single", device, Q.word_count(params))
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit, cached=True)
    # Length of the run, then replays at a few points of it.
    probe = Q.Generator(params, device=device)
    try:
        probe.seed()
        steps = probe.grow().steps
    finally:
        probe.close()
    stops = sorted({max(1, min(steps - 1, int(round(f * steps)))) for f in points}) if steps > 1 else []
    _, sms = _device_id(device)
    shapes = candidate_shapes(sms)
    timings = {s: [] for s in shapes}
    g = Q.Generator(params, device=device)
    try:
        g.seed()
        done = 0
        for stop in stops:
            st = g.grow(stop - done)
            done = stop
            if st.status != Q.QSGS_RUNNING:
                break
            for blocks, tile in shapes:
                g.set_grow_tile(tile)
                timings[(blocks, tile)].append(g.time_grow(blocks, reps))
    finally:
        g.close()
    if not all(timings.values()):
        best, timings = (0, 1), {}  # too short a run to time: the library default
    else:
        best = pick_best(timings)
    out = {"blocks": int(best[0]), "tile": int(best[1]),
           "timings_ms": {f"{b}x{t}": [round(x, 5) for x in v] for (b, t), v in timings.items()}}
    _store(key, out)
    return dict(out, cached=False)


def apply_single(gen: Q.Generator, shape: dict) -> None:
    gen.set_grow_blocks(shape["blocks"])
    gen.set_grow_tile(shape["tile"])


def tune_batch(params_list: list[dict], device=None, subset: int = 16, repeats: int = 2,
               use_cache: bool = True) -> dict:
    """Shape for batches like ``params_list``: each candidate runs a fixed
    subset of members from seeding to the end (``repeats`` times, the best
    counts: the first run of a shape builds its graph); returns {"blocks",
    "tile", "timings_ms", "cached"}."""
    import torch
    device = torch.device(device) if device is not None else torch.device(
        "cuda", torch.cuda.current_device())
    words_all = sum(Q.word_count(p) for p in params_list)
    key = cache_key("batch", device, words_all)
    if use_cache:
        hit = _load_cache().get(key)
        if hit:
            return dict(hit, cached=True)
    step = max(1, len(params_list) // subset)
    chosen = params_list[::step][:subset]
    words = sum(Q.word_count(p) for p in chosen)
    _, sms = _device_id(device)
    shapes = candidate_shapes(sms)
    timings = {s: [] for s in shapes}
    gens = [Q.Generator(p, device=device) for p in chosen]
    b = Q.Batch(len(chosen), words, device=device)
    try:
        b.set_members(gens)
        for blocks, tile in shapes:
            b.set_grow_blocks(blocks)
            b.set_grow_tile(tile)
            for _ in range(repeats):  # run() seeds every member again: the same work each time
                torch.cuda.synchronize(device)
                t0 = time.perf_counter()
                b.run()
                torch.cuda.synchronize(device)
                timings[(blocks, tile)].append((time.perf_counter() - t0) * 1e3)
    finally:
        b.close()
        for g in gens:
            g.close()
    # the best repeat of each shape (the first run of a shape builds its graph)
    timings = {s: [min(v)] for s, v in timings.items()}
    best = pick_best(timings)
    out = {"blocks": int(best[0]), "tile": int(best[1]), "members_timed": len(chosen),
           "timings_ms": {f"{b}x{t}": [round(x, 3) for x in v] for (b, t), v in timings.items()}}
    _store(key, out)
    return dict(out, cached=False)


def apply_batch(batch: Q.Batch, shape: dict) -> None:
    batch.set_grow_blocks(shape["blocks"])
    batch.set_grow_tile(shape["tile"])
