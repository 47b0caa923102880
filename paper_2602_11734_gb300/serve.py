"""Continuous-batching server for QSGS generation requests.

Requests (parameter dicts) arrive over time.  The server keeps every
admitted request's grid and candidate list resident on the GPU and advances
all of them together with one batch (``qsgs_batch_*``): each scheduling
round enqueues K growth steps of every running request as one CUDA graph
launch, and while the GPU works the host admits newly arrived requests --
as member slots, batch word space and the HBM budget allow -- and seeds them
on their own streams, so their seeding overlaps the running batch.  Finished
requests are trimmed to their exact target, copied to pinned host memory
and retired, freeing their memory for the queue.

Latency of a request = time from its arrival to its phase map being in host
memory.  Every request gets exactly the grid it gets alone.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

from . import qsgs as Q


@dataclass
class Request:
    rid: int
    params: dict
    arrival: float                      # seconds after the server clock starts
    voxels: int = 0
    admitted: float | None = None
    finished: float | None = None
    stats: Q.Stats | None = None
    result: object | None = None        # pinned host uint8 tensor (nz, ny, nx)
    rejected: str | None = None         # why it can never be admitted
    gen: Q.Generator | None = field(default=None, repr=False)

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


class Server:
    """Admission by free memory, resident state, interleaved steps."""

    def __init__(self, device=None, max_members: int = 256, max_words: int = 1 << 27,
                 hbm_budget: int | None = None, step_quantum: int = 8, keep_results: bool = True,
                 staging_voxels: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.batch = Q.Batch(max_members, max_words, device=self.device)
        self.max_members = max_members
        self.max_words = max_words
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(free * 0.8)
        self.hbm_budget = hbm_budget
        self.step_quantum = step_quantum
        self.keep_results = keep_results
        # Results that are not kept still land in host memory: one pinned
        # buffer, reused, sized for the largest request (grown on demand;
        # staging_voxels sizes it up front, outside any timed region).
        self._staging = None
        if staging_voxels:
            self._staging_buffer(staging_voxels)
        self.used_bytes = 0
        self.used_words = 0
        self.rounds = 0

    # -- admission ----------------------------------------------------------
    def _never_fits(self, r: Request) -> str | None:
        """Why the request cannot be admitted even into an empty server."""
        if Q.word_count(r.params) > self.max_words:
            return "more grid words than the batch word space"
        if Q.qsgs_workspace_bytes(r.params) > self.hbm_budget:
            return "workspace larger than the memory budget"
        return None

    def _fits(self, r: Request, n_members: int) -> bool:
        need = Q.qsgs_workspace_bytes(r.params)
        return (n_members < self.max_members and
                self.used_words + Q.word_count(r.params) <= self.max_words and
                self.used_bytes + need <= self.hbm_budget)

    def _admit(self, r: Request, now: float) -> None:
        r.gen = Q.Generator(r.params, device=self.device)
        r.gen.seed()                    # on the request's own stream
        r.admitted = now
        r.voxels = r.params["nx"] * r.params["ny"] * r.params["nz"]
        self.used_bytes += r.gen.nbytes
        self.used_words += Q.word_count(r.params)

    def _staging_buffer(self, voxels: int):
        torch = self.torch
        if self._staging is None or self._staging.numel() < voxels:
            self._staging = torch.empty(voxels, dtype=torch.uint8,
                                        pin_memory=torch.cuda.is_available())
        return self._staging

    def _retire(self, r: Request, st: Q.Stats, clock) -> None:
        torch = self.torch
        r.stats = st
        # The uint8 phase map goes to pinned host memory, written by the
        # device; the request finishes when it is there.
        if self.keep_results:
            host = torch.empty(r.gen.shape, dtype=torch.uint8, pin_memory=True)
            r.gen.fetch(out=host)
            r.result = host
        else:
            n = r.voxels
            r.gen.fetch(out=self._staging_buffer(n)[:n].view(r.gen.shape))
        r.finished = clock()
        self.used_bytes -= r.gen.nbytes
        self.used_words -= Q.word_count(r.params)
        r.gen.close()
        r.gen = None

    # -- main loop ----------------------------------------------------------
    def serve(self, requests: list[Request], timeout_s: float = 600.0) -> list[Request]:
        """Runs until every request is finished; arrivals are honoured in
        real time (requests are not admitted before their arrival).  A
        request that could not be admitted even into an empty server is
        marked ``rejected`` at once instead of holding up the queue."""
        for r in requests:
            r.rejected = self._never_fits(r)
        pending = sorted((r for r in requests if r.rejected is None), key=lambda r: r.arrival)
        running: list[Request] = []
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        qi = 0
        in_flight = False
        while qi < len(pending) or running:
            if clock() > timeout_s:
                raise TimeoutError("serving did not finish in time")
            # Admit what has arrived and fits (the batch may be running).
            joined = []
            while qi < len(pending) and pending[qi].arrival <= clock():
                r = pending[qi]
                if not self._fits(r, len(running) + len(joined)):
                    break
                self._admit(r, clock())
                joined.append(r)
                qi += 1
            finished = []
            if in_flight:
                stats = self.batch.query()        # waits for the round
                in_flight = False
                still = []
                for r, st in zip(running, stats):
                    if st.status == Q.QSGS_RUNNING:
                        still.append(r)
                    else:
                        finished.append((r, st))
                running = still
            if joined or len(running) != len(self.batch.members):
                running = running + joined
                self.batch.set_members([r.gen for r in running])
            if running:
                self.batch.advance(self.step_quantum)
                in_flight = True
                self.rounds += 1
            # The finished requests left the batch above; their maps are
            # fetched on their own streams while the next round runs.
            for r, st in finished:
                self._retire(r, st, clock)
            if not running and not finished and qi < len(pending):
                time.sleep(max(0.0, min(0.001, pending[qi].arrival - clock())))
        return requests


def summarize(requests: list[Request], wall_s: float | None = None) -> dict:
    """p50 / p99 latency, throughput in requests/s and nodes/s of the
    finished requests (rejected ones are counted apart)."""
    import numpy as np
    done = [r for r in requests if r.finished is not None]
    rejected = sum(1 for r in requests if r.rejected is not None)
    if not done:  # every request rejected (or none finished): no latency to report
        return {"requests": 0, "rejected": rejected, "p50_ms": None, "p99_ms": None,
                "mean_ms": None, "span_s": wall_s, "requests_per_s": None, "nodes_per_s": None}
    lat = np.array([r.latency for r in done])
    fin = max(r.finished for r in done)
    start = min(r.arrival for r in done)
    span = wall_s if wall_s is not None else fin - start
    voxels = sum(r.voxels for r in done)
    out = {"requests": len(done), "p50_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
           "span_s": span, "requests_per_s": len(done) / span,
           "nodes_per_s": voxels / span}
    if rejected:
        out["rejected"] = rejected
    return out
