"""Checkpoint and resume (qsgs_snapshot / qsgs_restore) through the C ABI: a
realization snapshotted after k steps, its handle destroyed and the snapshot
restored into a fresh handle and workspace, finishes with exactly the grid
and statistics of the uninterrupted run -- the oracle's grid, and at 400^3
the oracle-written golden.  What a step carries is the phase array, the
front, t and c_t (Sec. 2.3, Algorithm 3), and every draw is keyed by
(seed, voxel, t, direction)."""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2602_11734_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_11734_gb300 import build, qsgs
    build.build()
    qsgs.load_library()
    return qsgs


def resumed(Q, p, k, on_device):
    """Seed, grow k steps, snapshot, destroy; restore into a new handle and
    finish.  Returns (phase, stats, snapshot bytes)."""
    g = Q.Generator(p)
    g.seed()
    if k:
        g.grow(k)
    out = (torch.empty(Q.qsgs_snapshot_bytes(p), dtype=torch.uint8, device="cuda")
           if on_device else None)
    snap = g.snapshot(out)
    g.close()
    del g
    h = Q.Generator(p)
    try:
        h.restore(snap)
        st = h.grow()
        return h.fetch().cpu().numpy(), st, snap
    finally:
        h.close()


def uninterrupted(Q, p):
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow()
        return g.fetch().cpu().numpy(), st
    finally:
        g.close()


@pytest.mark.parametrize("case", [
    dict(),                                                  # 64^3, no spacing
    dict(nx=70, ny=33, nz=29, spacing_s=4, seed=5),          # ragged, spacing
    dict(nx=37, ny=29, nz=23, periodic=1, spacing_s=3, seed=9),  # torus
    dict(nx=40, ny=36, nz=33, g_face=1.0, g_edge=1.0, g_corner=1.0,
         target_solid_fraction=0.93),                        # exact-target trim
])
@pytest.mark.parametrize("k", [0, 1, 5, 17])
def test_resume_equals_uninterrupted_and_oracle(oracle, Q, case, k):
    p = dict(workloads.small_64(), **case)
    want = oracle.run(p)
    ref_phase, ref = uninterrupted(Q, p)
    for on_device in (False, True):
        phase, st, _ = resumed(Q, p, k, on_device)
        assert np.array_equal(phase, want.phase), (p, k, on_device)
        assert np.array_equal(phase, ref_phase)
        assert (st.solid_count, st.steps, st.status, st.front_size) == \
               (want.solid_count, want.steps, want.status, want.front_size)
        # the counters a step carries are restored, not recounted
        assert (st.sum_front, st.sum_draws, st.n_seeds, st.n_candidates) == \
               (ref.sum_front, ref.sum_draws, ref.n_seeds, ref.n_candidates)


def test_resume_of_a_finished_run(oracle, Q):
    p = dict(workloads.small_64(), nx=45, ny=41, nz=39, seed=3)
    g = Q.Generator(p)
    g.seed()
    st0 = g.grow()
    snap = g.snapshot()
    g.close()
    h = Q.Generator(p)
    try:
        h.restore(snap)
        assert h.query().status == st0.status == Q.QSGS_OK
        st = h.grow()
        assert (st.solid_count, st.steps, st.status) == (st0.solid_count, st0.steps, st0.status)
        assert np.array_equal(h.fetch().cpu().numpy(), oracle.run(p).phase)
    finally:
        h.close()


def test_resume_at_400_equals_the_golden(Q):
    with open(os.path.join(GOLDEN, "single_400.jsonl")) as f:
        row = json.loads(f.readline())
    p = row["params"]
    phase, st, snap = resumed(Q, p, 30, on_device=False)
    assert snap.numel() == 512 + 4 * 13 * 400 * 400
    assert hashlib.sha256(phase.tobytes()).hexdigest() == row["sha256_u8"]
    assert (st.solid_count, st.steps, st.status) == (row["solid_count"], row["steps"], row["status"])
    assert st.sum_front == sum(row["front_per_step"])


def test_restored_member_finishes_in_a_batch(oracle, Q):
    ps = [dict(workloads.small_64(), nx=50 + 3 * i, ny=47, nz=44, spacing_s=i, seed=20 + i)
          for i in range(3)]
    gens = []
    for i, p in enumerate(ps):
        g = Q.Generator(p)
        g.seed()
        g.grow(3 + i)
        snap = g.snapshot()
        g.close()
        h = Q.Generator(p)
        h.restore(snap)
        gens.append(h)
    b = Q.Batch(4, sum(Q.word_count(p) for p in ps))
    try:
        b.set_members(gens)
        b.advance()
        stats = b.query()
        for g, p, st in zip(gens, ps, stats):
            want = oracle.run(p)
            assert np.array_equal(g.fetch().cpu().numpy(), want.phase), p
            assert (st.solid_count, st.steps, st.status) == (want.solid_count, want.steps,
                                                             want.status)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_restore_rejects_foreign_or_damaged_snapshots(Q):
    p = dict(workloads.small_64(), nx=33, ny=20, nz=18)
    g = Q.Generator(p)
    try:
        with pytest.raises(Q.QsgsError) as e:
            g.snapshot()                          # not seeded yet
        assert e.value.code == Q.QSGS_ERR_STATE
        g.seed()
        g.grow(2)
        snap = g.snapshot()
        other = Q.Generator(dict(p, seed=p["seed"] + 1))
        try:
            with pytest.raises(Q.QsgsError) as e:
                other.restore(snap)               # another realization's snapshot
            assert e.value.code == Q.QSGS_ERR_INVALID
        finally:
            other.close()
        bad = snap.clone()
        bad[0] ^= 0xFF                            # not a snapshot
        with pytest.raises(Q.QsgsError) as e:
            g.restore(bad)
        assert e.value.code == Q.QSGS_ERR_INVALID
        with pytest.raises(Q.QsgsError) as e:
            g.restore(snap[:-4])                  # truncated
        assert e.value.code == Q.QSGS_ERR_INVALID
        with pytest.raises(Q.QsgsError) as e:
            g.snapshot(torch.empty(100, dtype=torch.uint8))  # too small
        assert e.value.code == Q.QSGS_ERR_INVALID
        g.restore(snap)                           # its own snapshot is fine
        g.grow()
    finally:
        g.close()
