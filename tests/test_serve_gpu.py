"""The continuous-batching server: requests that arrive while others run are
admitted as slots and memory free up, and every result equals the one the
request gets alone (the oracle's grid)."""
import numpy as np
import pytest

from paper_2602_11734_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_11734_gb300 import build, qsgs, serve
    build.build()
    qsgs.load_library()
    return serve


def requests(S, n, seed, spread_s):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        e = int(rng.integers(12, 48))
        p = dict(workloads.small_64(), nx=e, ny=int(rng.integers(12, 48)), nz=int(rng.integers(12, 48)),
                 cd=float(rng.choice([0.002, 0.01])), spacing_s=int(rng.integers(0, 7)),
                 target_solid_fraction=float(rng.uniform(0.5, 0.9)), seed=1000 + i)
        out.append(S.Request(rid=i, params=p, arrival=float(rng.uniform(0, spread_s))))
    return out


def test_every_served_result_equals_the_oracle(oracle, S):
    reqs = requests(S, 24, 1, 0.05)
    srv = S.Server(max_members=8, step_quantum=3)
    srv.serve(reqs)
    assert srv.rounds > 3
    for r in reqs:
        want = oracle.run(r.params)
        assert r.latency is not None and r.latency >= 0
        assert r.finished >= r.admitted >= r.arrival - 1e-6
        assert np.array_equal(r.result.numpy(), want.phase), r.params
        assert (r.stats.solid_count, r.stats.steps, r.stats.status) == \
               (want.solid_count, want.steps, want.status)
    summ = S.summarize(reqs)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_admission_waits_for_memory(oracle, S):
    from paper_2602_11734_gb300 import qsgs as Q
    reqs = requests(S, 12, 2, 0.0)      # all arrive at once
    biggest = max(Q.qsgs_workspace_bytes(r.params) for r in reqs)
    srv = S.Server(max_members=64, hbm_budget=2 * biggest, step_quantum=4)
    srv.serve(reqs)
    # at most two requests fit at a time, so admissions are spread out
    assert len({round(r.admitted, 6) for r in reqs}) > 3
    for r in reqs:
        assert np.array_equal(r.result.numpy(), oracle.run(r.params).phase)
