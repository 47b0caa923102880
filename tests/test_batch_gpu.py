"""Batched growth (many realizations per launch) against the oracle and the
single-realization path: every member must get exactly the grid and
statistics it gets alone, whatever the batch around it."""
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


def make_batch(Q, params, stream=None):
    gens = [Q.Generator(p) for p in params]
    words = sum(Q.word_count(p) for p in params)
    b = Q.Batch(max(1, len(params)), words, stream=stream)
    b.set_members(gens)
    return b, gens


def check_member(oracle, g, st, p):
    want = oracle.run(p)
    got = g.fetch().cpu().numpy()
    assert np.array_equal(got, want.phase), p
    assert (st.solid_count, st.steps, st.status, st.front_size, st.n_seeds) == \
           (want.solid_count, want.steps, want.status, want.front_size, want.n_accepted), p
    if want.log is not None and want.log.size:
        assert st.sum_front == int(want.log["front"].sum()), p


def test_batch_of_uneven_small_realizations(oracle, Q):
    rng = np.random.default_rng(99)
    params = [workloads.random_small(rng, max_edge=26) for _ in range(14)]
    params.append(dict(workloads.small_64()))
    b, gens = make_batch(Q, params)
    try:
        stats = b.run()
        for g, st, p in zip(gens, stats, params):
            check_member(oracle, g, st, p)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_batch_at_the_member_limit(oracle, Q):
    # 1024 members (the most a batch takes): one control thread and one
    # state-gather block per member.  Each member must match the oracle, and
    # the batch's gathered statistics must equal each handle's own query.
    rng = np.random.default_rng(4242)
    params = [workloads.random_small(rng, max_edge=12) for _ in range(1024)]
    b, gens = make_batch(Q, params)
    try:
        stats = b.run()
        assert len(stats) == 1024
        for g, st, p in zip(gens, stats, params):
            check_member(oracle, g, st, p)
            own = g.query()
            assert (own.solid_count, own.steps, own.status, own.front_size, own.sum_front) == \
                   (st.solid_count, st.steps, st.status, st.front_size, st.sum_front), p
    finally:
        b.close()
        for g in gens:
            g.close()


def test_batch_equals_single_path(Q):
    params = [dict(workloads.single_400(), nx=e, ny=e - 3, nz=e + 5, seed=s,
                   target_solid_fraction=0.7 + 0.02 * s)
              for s, e in enumerate((48, 64, 80, 33, 97))]
    singles = []
    for p in params:
        out, st = Q.generate(p)
        singles.append((hashlib.sha256(out.cpu().numpy().tobytes()).hexdigest(), st))
    b, gens = make_batch(Q, params)
    try:
        stats = b.run()
        for g, st, (h, s1) in zip(gens, stats, singles):
            assert hashlib.sha256(g.fetch().cpu().numpy().tobytes()).hexdigest() == h
            assert (st.solid_count, st.steps, st.status, st.front_size, st.sum_front) == \
                   (s1.solid_count, s1.steps, s1.status, s1.front_size, s1.sum_front)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_membership_changes_mid_run(oracle, Q):
    rng = np.random.default_rng(7)
    params = [dict(workloads.small_64(), nx=int(rng.integers(20, 50)), ny=int(rng.integers(20, 50)),
                   nz=int(rng.integers(20, 50)), spacing_s=int(rng.integers(0, 6)), seed=i)
              for i in range(5)]
    gens = [Q.Generator(p) for p in params]
    words = sum(Q.word_count(p) for p in params)
    b = Q.Batch(5, words)
    try:
        for g in gens:
            g.seed()
        a, bb, c, d, e = gens
        b.set_members([a, bb, c])
        b.advance(3)
        b.query()
        b.set_members([bb, c, d])       # a leaves, d joins fresh
        b.advance(4)
        b.query()
        a.grow(2)                       # a continues alone for a while
        b.set_members([d, a, e, bb])    # a rejoins, e joins, c leaves
        b.advance(0)
        stats = {id(x): s for x, s in zip(b.members, b.query())}
        c_st = c.grow()                 # c finishes alone
        for g, p in zip(gens, params):
            st = c_st if g is c else stats[id(g)]
            check_member(oracle, g, st, p)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_domain_kind_switches_between_advances(oracle, Q):
    # Open-only memberships run the open-domain growth kernel, memberships
    # with a periodic member the run-time one; the batch graph is rebuilt
    # whenever the kind changes, mid-run included.
    rng = np.random.default_rng(11)
    opens = [dict(workloads.small_64(), nx=int(rng.integers(20, 45)), ny=int(rng.integers(20, 45)),
                  nz=int(rng.integers(20, 45)), spacing_s=int(rng.integers(0, 5)), seed=30 + i)
             for i in range(3)]
    torus = dict(workloads.small_64(), nx=33, ny=29, nz=31, spacing_s=3, seed=41, periodic=1)
    params = opens + [torus]
    gens = [Q.Generator(p) for p in params]
    b = Q.Batch(4, sum(Q.word_count(p) for p in params))
    try:
        for g in gens:
            g.seed()
        o1, o2, o3, per = gens
        b.set_members([o1, o2])           # open only
        b.advance(3)
        b.query()
        b.set_members([o1, per, o3])      # a periodic member joins: run-time kind
        b.advance(3)
        b.query()
        b.set_members([o2, o3])           # open only again
        b.advance(0)
        stats = {id(x): s for x, s in zip(b.members, b.query())}
        b.set_members([o1, per])          # mixed, to the end
        b.advance(0)
        stats.update({id(x): s for x, s in zip(b.members, b.query())})
        for g, p in zip(gens, params):
            check_member(oracle, g, stats[id(g)], p)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_batch_rerun_and_direct_launches(oracle, Q):
    rng = np.random.default_rng(5)
    params = [workloads.random_small(rng, max_edge=30) for _ in range(6)]
    b, gens = make_batch(Q, params)
    try:
        b.run()
        first = [g.fetch().clone() for g in gens]
        b.set_profiling(True)           # direct launches instead of the graph
        stats = b.run()
        prof = b.profile()
        for g, f, st, p in zip(gens, first, stats, params):
            assert torch.equal(g.fetch(), f)
            check_member(oracle, g, st, p)
        assert prof["grow"][0] >= 1
    finally:
        b.close()
        for g in gens:
            g.close()


def test_batch_96_instances_golden(Q):
    path = os.path.join(GOLDEN, "batch_96.jsonl")
    if not os.path.exists(path):
        pytest.skip("batch_96 golden not generated")
    rows = [json.loads(line) for line in open(path)]
    params = [r["params"] for r in rows]
    b, gens = make_batch(Q, params)
    try:
        stats = b.run()
        for g, st, row in zip(gens, stats, rows):
            phase = g.fetch().cpu().numpy()
            assert hashlib.sha256(phase.tobytes()).hexdigest() == row["sha256_u8"], row["params"]
            assert (st.solid_count, st.steps, st.status, st.front_size) == \
                   (row["solid_count"], row["steps"], row["status"], row["front_size"])
            assert st.sum_front == sum(row["front_per_step"])
    finally:
        b.close()
        for g in gens:
            g.close()


def test_batch_tile_and_grid_do_not_change_results(oracle, Q, tmp_path, monkeypatch):
    from paper_2602_11734_gb300 import tune
    monkeypatch.setenv("QSGS_TUNE_CACHE", str(tmp_path / "tune.json"))
    rng = np.random.default_rng(11)
    params = [workloads.random_small(rng, max_edge=28) for _ in range(6)]
    shape = tune.tune_batch(params, subset=3, repeats=1)
    assert shape["members_timed"] == 3 and not shape["cached"]
    for blocks, tile in ((shape["blocks"], shape["tile"]), (40, 16)):
        b, gens = make_batch(Q, params)
        try:
            tune.apply_batch(b, {"blocks": blocks, "tile": tile})
            stats = b.run()
            for g, st, p in zip(gens, stats, params):
                check_member(oracle, g, st, p)
        finally:
            b.close()
            for g in gens:
                g.close()


def test_batch_reseed_follows_member_settings(oracle, Q):
    # Repeated seeding of the same members replays one captured graph; a
    # member whose settings change (here its cells of an earlier phase) must
    # be seeded from the new settings, and again after they are removed.
    rng = np.random.default_rng(515)
    params = [dict(workloads.random_small(rng, max_edge=24), cd=0.03, max_steps=0)
              for _ in range(5)]
    p0 = params[0]
    shape = (p0["nz"], p0["ny"], p0["nx"])
    blk = rng.random(shape) < 0.3
    words = (p0["nx"] + 31) // 32
    packed = np.zeros((p0["nz"], p0["ny"], words * 32), dtype=bool)
    packed[:, :, :p0["nx"]] = blk
    w32 = np.packbits(packed, axis=-1, bitorder="little").view(np.uint32).reshape(-1)
    t = torch.from_numpy(w32.view(np.int32).copy()).cuda()
    b, gens = make_batch(Q, params)
    try:
        prev = None
        for blocked in (None, None, blk, blk, None):  # capture, replay, capture, replay, capture
            if blocked is not prev:
                gens[0].set_blocked(None if blocked is None else t)
                prev = blocked
            b.set_members(gens)
            stats = b.run()
            for k, (g, st, p) in enumerate(zip(gens, stats, params)):
                want = oracle.run(p, blocked=blocked if k == 0 else None)
                assert np.array_equal(g.fetch().cpu().numpy(), want.phase), (k, p)
                assert (st.solid_count, st.steps, st.front_size) == \
                       (want.solid_count, want.steps, want.front_size), (k, p)
    finally:
        b.close()
        for g in gens:
            g.close()
