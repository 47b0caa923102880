"""Host logic of the continuous-batching server on the CPU: the scheduling
loop of ``Server.serve`` driven with stand-ins for the generator and the
batch (no device), checking admission by arrival time, member slots, batch
word space and memory budget, requests joining a running batch, and
retirement after exactly the steps each request needs."""
import time
from types import SimpleNamespace

import pytest

torch = pytest.importorskip("torch")

from paper_2602_11734_gb300 import qsgs as Q  # noqa: E402
from paper_2602_11734_gb300 import serve as S  # noqa: E402


class Log:
    def __init__(self):
        self.rounds = []      # member lists, one per advance
        self.joins_mid_run = 0


def make_fakes(log: Log, max_members: int, max_words: int, budget: int):
    class FakeGen:
        def __init__(self, params, device=None):
            self.params = params
            self.need = 1 + params["seed"] % 7          # steps this request takes
            self.done = 0
            self.seeded = self.closed = self.fetched = False
            self.nbytes = Q.qsgs_workspace_bytes(params)
            self.words = Q.word_count(params)
            self.shape = (params["nz"], params["ny"], params["nx"])

        def seed(self):
            self.seeded = True
            self.done = 0

        def fetch(self, fmt="u8", out=None):
            assert self.done == self.need and not self.closed
            self.fetched = True

        def close(self):
            self.closed = True

    class FakeBatch:
        def __init__(self, n, words, device=None):
            assert (n, words) == (max_members, max_words)
            self.members = []

        def set_members(self, gens):
            assert len(gens) <= max_members
            assert sum(g.words for g in gens) <= max_words
            assert sum(g.nbytes for g in gens) <= budget
            assert all(g.seeded and not g.closed for g in gens)
            if any(g.done > 0 for g in gens) and any(g.done == 0 for g in gens):
                log.joins_mid_run += 1
            self.members = list(gens)

        def advance(self, k):
            assert self.members
            log.rounds.append(list(self.members))
            for g in self.members:
                g.done = min(g.need, g.done + k)

        def query(self):
            time.sleep(0.003)  # the round's device time: later arrivals queue meanwhile
            return [SimpleNamespace(status=Q.QSGS_RUNNING if g.done < g.need else Q.QSGS_OK)
                    for g in self.members]

    return FakeGen, FakeBatch


def params(i: int, edge: int) -> dict:
    return dict(nx=edge, ny=edge, nz=edge, cd=1e-3, g_face=0.01, g_edge=0.0025,
                g_corner=0.000625, spacing_s=0, target_solid_fraction=0.5, target_count=0,
                seed=i, max_steps=0)


@pytest.mark.parametrize("max_members, budget_requests", [(3, 100), (16, 2), (16, 100)])
def test_server_schedules_requests_within_its_limits(monkeypatch, max_members, budget_requests):
    edges = [32, 48, 64, 40, 32, 56, 64, 36, 44, 32, 60, 48]
    reqs = [S.Request(rid=i, params=params(i, e), arrival=0.002 * i) for i, e in enumerate(edges)]
    biggest = max(Q.qsgs_workspace_bytes(r.params) for r in reqs)
    budget = budget_requests * biggest
    max_words = 1 << 20
    log = Log()
    gen_cls, batch_cls = make_fakes(log, max_members, max_words, budget)
    monkeypatch.setattr(Q, "Generator", gen_cls)
    monkeypatch.setattr(Q, "Batch", batch_cls)
    srv = S.Server(device="cuda:0", max_members=max_members, max_words=max_words,
                   hbm_budget=budget, step_quantum=2, keep_results=False)
    done = srv.serve(reqs, timeout_s=30.0)
    assert done is reqs
    for r in reqs:
        assert r.admitted is not None and r.admitted >= r.arrival      # not before arrival
        assert r.finished is not None and r.finished >= r.admitted
        assert r.latency == pytest.approx(r.finished - r.arrival)
        assert r.gen is None and r.voxels == r.params["nx"] ** 3
    # every request ran exactly the steps it needs, was fetched and closed
    seen = {id(g): g for rnd in log.rounds for g in rnd}
    assert len(seen) == len(reqs)
    assert all(g.done == g.need and g.fetched and g.closed for g in seen.values())
    # a finished member is never advanced again after it was retired
    for rnd in log.rounds:
        assert all(g.done <= g.need for g in rnd)
    assert srv.used_bytes == 0 and srv.used_words == 0
    assert srv.rounds == len(log.rounds)
    if max_members > 3 and budget_requests > 2:
        assert log.joins_mid_run > 0    # continuous batching: joins while others run
    assert max(len(rnd) for rnd in log.rounds) <= max_members
    s = S.summarize(reqs)
    assert s["requests"] == len(reqs) and s["p50_ms"] <= s["p99_ms"]
    assert s["nodes_per_s"] > 0


@pytest.mark.parametrize("limit", ["budget", "words"])
def test_a_request_that_can_never_fit_is_rejected_at_once(monkeypatch, limit):
    # Larger than the memory budget or the batch word space even for an
    # empty server: rejected on entry instead of holding up the queue.
    log = Log()
    small, big = params(0, 32), params(1, 128)
    budget = Q.qsgs_workspace_bytes(small) if limit == "budget" else 1 << 40
    max_words = 1 << 20 if limit == "budget" else Q.word_count(small)
    gen_cls, batch_cls = make_fakes(log, 4, max_words, budget)
    monkeypatch.setattr(Q, "Generator", gen_cls)
    monkeypatch.setattr(Q, "Batch", batch_cls)
    srv = S.Server(device="cuda:0", max_members=4, max_words=max_words, hbm_budget=budget,
                   step_quantum=2, keep_results=False)
    reqs = [S.Request(rid=0, params=small, arrival=0.0),
            S.Request(rid=1, params=big, arrival=0.0),
            S.Request(rid=2, params=params(2, 32), arrival=0.001)]
    srv.serve(reqs, timeout_s=5.0)
    assert reqs[1].rejected and reqs[1].admitted is None and reqs[1].finished is None
    assert all(r.rejected is None and r.finished is not None for r in (reqs[0], reqs[2]))
    s = S.summarize(reqs)
    assert s["requests"] == 2 and s["rejected"] == 1


def test_summary_when_every_request_is_rejected(monkeypatch):
    # No finished request: the summary reports the rejections and no
    # latency or rate instead of failing on an empty set.
    log = Log()
    small, big = params(0, 32), params(1, 128)
    budget = Q.qsgs_workspace_bytes(small)
    gen_cls, batch_cls = make_fakes(log, 4, 1 << 20, budget)
    monkeypatch.setattr(Q, "Generator", gen_cls)
    monkeypatch.setattr(Q, "Batch", batch_cls)
    srv = S.Server(device="cuda:0", max_members=4, max_words=1 << 20, hbm_budget=budget,
                   step_quantum=2, keep_results=False)
    reqs = [S.Request(rid=i, params=dict(big, seed=i), arrival=0.0) for i in range(3)]
    srv.serve(reqs, timeout_s=5.0)
    assert all(r.rejected and r.finished is None for r in reqs)
    assert log.rounds == []
    s = S.summarize(reqs)
    assert s["requests"] == 0 and s["rejected"] == 3
    assert s["p50_ms"] is None and s["p99_ms"] is None and s["requests_per_s"] is None


def test_next_round_starts_before_finished_maps_are_fetched(monkeypatch):
    # After a round, requests that finished leave the batch and the next
    # round is launched first; their maps are fetched while it runs.  So
    # between the query that found a request done and its fetch there is an
    # advance whenever other requests were still running.
    log = Log()
    events = []
    gen_cls, batch_cls = make_fakes(log, 8, 1 << 20, 1 << 40)

    class Gen(gen_cls):
        def fetch(self, fmt="u8", out=None):
            super().fetch(fmt, out)
            events.append(("fetch", id(self)))

    class Batch(batch_cls):
        def advance(self, k):
            super().advance(k)
            events.append(("advance", None))

        def query(self):
            out = super().query()
            running = sum(1 for s in out if s.status == Q.QSGS_RUNNING)
            events.append(("query", running))
            return out

    monkeypatch.setattr(Q, "Generator", Gen)
    monkeypatch.setattr(Q, "Batch", Batch)
    srv = S.Server(device="cuda:0", max_members=8, max_words=1 << 20, hbm_budget=1 << 40,
                   step_quantum=1, keep_results=False)
    # different step counts (1 + seed % 7), all present from the start
    reqs = [S.Request(rid=i, params=params(i, 32), arrival=0.0) for i in range(6)]
    srv.serve(reqs, timeout_s=30.0)
    assert all(r.finished is not None for r in reqs)
    checked = 0
    for i, (kind, _) in enumerate(events):
        if kind != "fetch":
            continue
        q = max(j for j in range(i) if events[j][0] == "query")
        if events[q][1] > 0:  # others still running after that round
            assert any(events[j][0] == "advance" for j in range(q + 1, i)), events[q:i + 1]
            checked += 1
    assert checked > 0
