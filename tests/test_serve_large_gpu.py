"""The served configuration at its real sizes.  The large requests of the
2000-request mix -- the first three of each of the edges 256, 400 and 512
-- go through the continuous-batching server while the small requests of
the mix arrive and run beside them, and each large request runs once more
alone on the single-realization path.  Every result, in the mix and alone,
equals the oracle-written golden: SHA-256 of the uint8 phase map, solid
count, steps and status."""
import hashlib
import json
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    with open(os.path.join(GOLDEN, f"{name}.jsonl")) as f:
        return [json.loads(line) for line in f]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_11734_gb300 import build, qsgs, serve
    build.build()
    qsgs.load_library()
    return serve


def check(row, phase_bytes, st, where):
    assert hashlib.sha256(phase_bytes).hexdigest() == row["sha256_u8"], (where, row["params"])
    assert (st.solid_count, st.steps, st.status) == \
           (row["solid_count"], row["steps"], row["status"]), (where, row["params"])


def test_large_requests_in_the_mix_and_alone_equal_the_golden(S):
    from paper_2602_11734_gb300 import qsgs as Q
    large, small = rows("serve_large"), rows("serve_small")
    assert sorted({r["params"]["nx"] for r in large}) == [256, 400, 512] and len(large) == 9
    reqs = []
    # Large requests every 20 ms; small ones spread over the same 300 ms, so
    # they arrive while the large ones run and join the running batch.
    for i, r in enumerate(large):
        reqs.append((r, S.Request(rid=i, params=r["params"], arrival=0.02 * i)))
    for j, r in enumerate(small):
        reqs.append((r, S.Request(rid=100 + j, params=r["params"], arrival=0.3 * j / len(small))))
    srv = S.Server(max_members=64, step_quantum=4)
    srv.serve([q for _, q in reqs])
    assert srv.rounds > 5
    # Continuous batching: some small request was admitted while a large
    # one was still running.
    first_large_done = min(q.finished for r, q in reqs if q.rid < 100)
    assert any(q.admitted < first_large_done for r, q in reqs if q.rid >= 100)
    for r, q in reqs:
        check(r, q.result.numpy().tobytes(), q.stats, "in the mix")
    # The same large requests alone.
    for r in large:
        g = Q.Generator(r["params"])
        try:
            g.seed()
            st = g.grow()
            host = torch.empty(g.shape, dtype=torch.uint8, pin_memory=True)
            g.fetch(out=host)
            check(r, host.numpy().tobytes(), st, "alone")
        finally:
            g.close()
