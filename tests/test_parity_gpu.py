"""GPU path (through the C ABI) against the CPU oracle, voxel for voxel.

Every case compares the full phase map and the run summary (solid count,
steps, status, front size, candidates, seeds) bit-exactly: the method is
integer arithmetic end to end, so there is no tolerance.
"""
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


def gpu_run(Q, p, chunk=0):
    g = Q.Generator(p)
    try:
        g.seed()
        if chunk:
            while True:
                st = g.grow(chunk)
                if st.status != Q.QSGS_RUNNING:
                    break
        else:
            st = g.grow()
        phase = g.fetch().cpu().numpy()
        packed = g.fetch(fmt="packed").cpu().numpy().view(np.uint32)
        return phase, packed, st
    finally:
        g.close()


def assert_same(oracle, Q, p, chunk=0):
    want = oracle.run(p)
    phase, packed, st = gpu_run(Q, p, chunk)
    mism = np.flatnonzero(phase.ravel() != want.phase.ravel())
    assert mism.size == 0, (p, mism[:10], mism.size)
    assert st.solid_count == want.solid_count, p
    assert st.target_count == want.target_count, p
    assert st.steps == want.steps, p
    assert st.status == want.status, p
    assert st.front_size == want.front_size, p
    assert st.n_candidates == want.n_candidates, p
    assert st.n_seeds == want.n_accepted, p
    if want.log is not None and want.log.size:
        assert st.sum_front == int(want.log["front"].sum()), p
    # the packed format holds the same voxels
    nz, ny, nx = phase.shape
    W = (nx + 31) // 32
    bits = np.unpackbits(packed.view(np.uint8), bitorder="little").reshape(nz, ny, W * 32)
    assert np.array_equal(bits[:, :, :nx], phase)
    assert not bits[:, :, nx:].any()
    return want, st


def test_small_64_parity(oracle, Q):
    assert_same(oracle, Q, workloads.small_64())


def test_random_small_parity(oracle, Q):
    rng = np.random.default_rng(1234)
    for _ in range(60):
        assert_same(oracle, Q, workloads.random_small(rng, max_edge=24))


@pytest.mark.parametrize("dims", [(70, 33, 29), (97, 5, 41), (33, 64, 17), (129, 31, 9),
                                  (1, 200, 30), (200, 1, 1), (31, 32, 33), (64, 1, 64)])
def test_ragged_multiword_parity(oracle, Q, dims):
    nx, ny, nz = dims
    for s, cd in ((0, 0.004), (4, 0.01), (9, 0.02)):
        p = dict(workloads.small_64(), nx=nx, ny=ny, nz=nz, spacing_s=s, cd=cd,
                 seed=nx * 7919 + s)
        assert_same(oracle, Q, p)


@pytest.mark.parametrize("extra", [
    dict(nx=1, ny=1, nz=1, cd=1.0, target_solid_fraction=1.0),
    dict(nx=1, ny=1, nz=1, cd=0.0, target_solid_fraction=1.0),
    dict(cd=0.0),                                                   # no seeds: stalled
    dict(cd=1.0, target_solid_fraction=1.0),                        # all seeds
    dict(cd=0.3, target_count=17),                                  # seed cap
    dict(g_face=0.0, g_edge=0.0, g_corner=0.0),                     # G = 0: stalled
    dict(g_face=1.0, g_edge=1.0, g_corner=1.0, target_solid_fraction=0.93),  # G = 1, trim
    dict(g_face=0.0, g_edge=1.0, g_corner=0.0, cd=0.0005, target_solid_fraction=0.9),
    dict(target_solid_fraction=0.0),
    dict(target_solid_fraction=1.0, max_steps=7),
    dict(max_steps=1),
    dict(spacing_s=1),
    dict(spacing_s=64, cd=0.05),
    dict(seed=2**64 - 1),
    # dense fronts: thousands of (voxel, block) pairs per 32-word chunk and
    # half of the draws passing (the claim buffer flushes every iteration)
    dict(cd=0.35, g_face=0.5, g_edge=0.5, g_corner=0.5, target_solid_fraction=0.97),
    dict(cd=0.3, g_face=0.004, g_edge=0.004, g_corner=0.004, target_solid_fraction=0.97),  # 16 steps
    dict(cd=0.12, g_face=1.0, g_edge=1.0, g_corner=1.0, target_solid_fraction=0.99, periodic=1),
])
def test_edge_case_parity(oracle, Q, extra):
    p = dict(workloads.small_64(), nx=37, ny=29, nz=23)
    p.update(extra)
    assert_same(oracle, Q, p)


@pytest.mark.parametrize("s", [8, 10])
def test_dense_conflict_lists_parity(oracle, Q, s):
    """Dense candidates (cd = 0.02 on 64^3, about 5.2 k of them) with
    27 k (s = 8) and 53 k (s = 10) earlier conflicts: long conflict lists
    for the spacing rounds, whose decisions stay in shared memory."""
    p = dict(workloads.small_64(), cd=0.02, spacing_s=s, seed=11 + s)
    assert_same(oracle, Q, p)


def test_chunked_growth_equals_one_shot(oracle, Q):
    p = dict(workloads.small_64(), nx=48, ny=40, nz=36, spacing_s=3)
    for chunk in (1, 3, 5):
        assert_same(oracle, Q, p, chunk=chunk)


def test_repeat_and_reseed_are_deterministic(Q):
    p = dict(workloads.small_64(), nx=90, ny=70, nz=50, spacing_s=6)
    g = Q.Generator(p)
    try:
        g.seed()
        g.grow()
        a = g.fetch().clone()
        g.seed()  # restart the same realization in the same workspace
        g.grow()
        b = g.fetch()
        assert torch.equal(a, b)
    finally:
        g.close()


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.jsonl")
    if not os.path.exists(path):
        pytest.skip(f"{name} golden not generated")
    return [json.loads(line) for line in open(path)]


def _check_golden_row(Q, row):
    phase, _, st = gpu_run(Q, row["params"])
    assert hashlib.sha256(phase.tobytes()).hexdigest() == row["sha256_u8"], row["params"]
    assert st.solid_count == row["solid_count"]
    assert st.steps == row["steps"]
    assert st.status == row["status"]
    assert st.front_size == row["front_size"]
    assert st.n_candidates == row["n_candidates"]
    assert st.n_seeds == row["n_accepted"]
    assert st.sum_front == sum(row["front_per_step"])


def test_single_400_golden(Q):
    for row in _golden("single_400"):
        _check_golden_row(Q, row)


def test_sweep_500_golden(Q):
    for row in _golden("sweep_500"):
        _check_golden_row(Q, row)


def test_batch_96_instances_golden(Q):
    for row in _golden("batch_96"):
        _check_golden_row(Q, row)


def test_serve_small_golden(Q):
    for row in _golden("serve_small"):
        _check_golden_row(Q, row)


def test_direct_launch_path_matches_graph_path(oracle, Q):
    # The event profiler forces direct launches (no CUDA graph); both paths
    # must give the oracle's grid.
    p = dict(workloads.small_64(), nx=61, ny=47, nz=39, spacing_s=5, cd=0.006)
    want = oracle.run(p)
    g = Q.Generator(p)
    try:
        g.set_profiling(True)
        g.seed()
        st = g.grow()
        prof = g.profile()
        got = g.fetch().cpu().numpy()
    finally:
        g.close()
    assert np.array_equal(got, want.phase)
    assert (st.solid_count, st.steps, st.status) == (want.solid_count, want.steps, want.status)
    assert prof["grow"][0] >= st.steps and prof["grow"][1] > 0


def test_legacy_default_stream(oracle, Q):
    class NullStream:
        cuda_stream = 0
    p = dict(workloads.small_64(), nx=33, ny=35, nz=37, spacing_s=2)
    want = oracle.run(p)
    g = Q.Generator(p, stream=NullStream())
    try:
        g.seed()
        st = g.grow()
        got = g.fetch().cpu().numpy()
    finally:
        g.close()
    assert np.array_equal(got, want.phase)
    assert st.steps == want.steps


def test_launch_counter_grows_with_steps(Q):
    p = dict(workloads.small_64(), nx=50, ny=50, nz=50)
    g = Q.Generator(p)
    try:
        g.seed()
        before = g.query().launches
        st = g.grow()
        assert st.launches - before >= 3 * st.steps
    finally:
        g.close()


def test_philox_probe_and_draw_counter(Q):
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    ms = Q.qsgs_bench_philox(1 << 24, out.data_ptr(), 0)
    assert ms > 0 and int(out.item()) != 0
    p = dict(workloads.small_64(), nx=40, ny=40, nz=40)
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow()
        # at least one Philox block per growth step, at most 7 per front voxel
        assert st.steps <= st.sum_draws <= 7 * st.sum_front
    finally:
        g.close()


def test_time_grow_probe_leaves_the_run_unchanged(oracle, Q):
    p = dict(workloads.small_64(), nx=72, ny=70, nz=68, spacing_s=4)
    want = oracle.run(p)
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow(5)
        assert st.status == Q.QSGS_RUNNING
        for blocks in (0, 64, 1000):
            assert g.time_grow(blocks, reps=3) > 0
        g.grow(3)
        assert g.time_grow(0, reps=2) > 0
        st = g.grow()
        assert np.array_equal(g.fetch().cpu().numpy(), want.phase)
        assert (st.solid_count, st.steps, st.status, st.sum_front) == \
               (want.solid_count, want.steps, want.status, int(want.log["front"].sum()))
    finally:
        g.close()


def test_autotuned_shape_keeps_results(oracle, Q, tmp_path, monkeypatch):
    from paper_2602_11734_gb300 import tune
    monkeypatch.setenv("QSGS_TUNE_CACHE", str(tmp_path / "tune.json"))
    p = dict(workloads.small_64(), nx=96, ny=90, nz=88, spacing_s=5, seed=17)
    shape = tune.tune_single(p, reps=2)
    assert not shape["cached"] and shape["tile"] in tune.TILES
    assert len(shape["timings_ms"]) == len(tune.candidate_shapes(torch.cuda.get_device_properties(0).multi_processor_count))
    assert tune.tune_single(p)["cached"]
    want = oracle.run(p)
    for blocks, tile in ((shape["blocks"], shape["tile"]), (152, 8), (0, 3)):
        g = Q.Generator(p)
        try:
            tune.apply_single(g, {"blocks": blocks, "tile": tile})
            g.seed()
            st = g.grow()
            assert np.array_equal(g.fetch().cpu().numpy(), want.phase), (blocks, tile)
            assert (st.solid_count, st.steps, st.sum_front) == \
                   (want.solid_count, want.steps, int(want.log["front"].sum()))
        finally:
            g.close()


def test_host_u8_fetch_in_slabs(oracle, Q):
    # A pageable host buffer is staged through the candidate-list area, which
    # is smaller than the grid in bytes: several slabs, ragged last one.
    p = dict(workloads.small_64(), nx=77, ny=45, nz=61, cd=0.001, spacing_s=4, seed=23)
    assert Q.word_count(p) * 4 < p["nx"] * p["ny"] * p["nz"]
    want = oracle.run(p)
    g = Q.Generator(p)
    try:
        g.seed()
        g.grow()
        host = torch.empty(g.shape, dtype=torch.uint8)
        assert not host.is_pinned()
        g.fetch(out=host)
        dev = g.fetch()
        assert np.array_equal(host.numpy(), want.phase)
        assert torch.equal(dev.cpu(), host)
    finally:
        g.close()


def test_host_u8_fetch_into_mapped_memory(oracle, Q):
    # Pinned host memory is written by the device directly, mid-run too; the
    # same flag on pageable memory falls back to the staged copy.
    p = dict(workloads.small_64(), nx=77, ny=45, nz=61, cd=0.001, spacing_s=4, seed=29)
    n = p["nx"] * p["ny"] * p["nz"]
    g = Q.Generator(p)
    try:
        g.seed()
        g.grow(3)
        mid = torch.full(g.shape, 7, dtype=torch.uint8, pin_memory=True)
        g.fetch(out=mid)                                   # running: direct writes
        assert torch.equal(mid, g.fetch().cpu())
        g.grow()
        host = torch.full(g.shape, 7, dtype=torch.uint8, pin_memory=True)
        Q.qsgs_fetch(g.handle, host.data_ptr(), n, Q.QSGS_FMT_U8, Q.QSGS_DST_HOST_MAPPED)
        assert np.array_equal(host.numpy(), oracle.run(p).phase)
        pageable = torch.full(g.shape, 7, dtype=torch.uint8)
        Q.qsgs_fetch(g.handle, pageable.data_ptr(), n, Q.QSGS_FMT_U8, Q.QSGS_DST_HOST_MAPPED)
        assert torch.equal(pageable, host)
        with pytest.raises(Q.QsgsError):
            Q.qsgs_fetch(g.handle, host.data_ptr(), n, Q.QSGS_FMT_U8, 3)  # no such kind
    finally:
        g.close()


@pytest.mark.parametrize("spacing", [True, False])
def test_fig3_setting_small(oracle, Q, spacing):
    # The size sweep's parameters (one G_ref for every class) on a small box.
    p = dict(workloads.fig3_size(72, spacing), ny=66, nz=70)
    want = oracle.run(p)
    out, st = Q.generate(p)
    assert np.array_equal(out.cpu().numpy(), want.phase)
    assert (st.solid_count, st.steps, st.status) == (want.solid_count, want.steps, want.status)


@pytest.mark.parametrize("case", [dict(nx=70, ny=66, nz=61, spacing_s=4, seed=3),
                                  dict(nx=33, ny=90, nz=40, spacing_s=0, seed=8, cd=0.004)])
def test_fullfield_comparator_is_the_same_realization(oracle, Q, case):
    # Algorithm 2's full-field sweep on the same keyed draws == Algorithm 3.
    p = dict(workloads.small_64(), **case)
    want = oracle.run(p)
    lists = Q.Generator(p)
    full = Q.Generator(p)
    try:
        lists.seed()
        a = lists.grow()
        full.set_mode(Q.QSGS_MODE_FULLFIELD)
        full.seed()
        half = full.grow(max(1, want.steps // 2))  # switch modes mid-run as well
        full.set_mode(Q.QSGS_MODE_LIETS)
        full.grow(2)
        full.set_mode(Q.QSGS_MODE_FULLFIELD)
        b = full.grow()
        assert half.status == Q.QSGS_RUNNING
        assert np.array_equal(full.fetch().cpu().numpy(), want.phase)
        assert torch.equal(full.fetch(), lists.fetch())
        assert (b.solid_count, b.steps, b.status, b.sum_front, b.front_size) == \
               (a.solid_count, a.steps, a.status, a.sum_front, a.front_size)
        assert b.sum_draws > a.sum_draws  # every voxel drew every block
    finally:
        lists.close()
        full.close()


def test_fontainebleau_setting_small(oracle, Q):
    # The Sec. 3.3 parameterisation (S_d from the grain diameter, one G_ref)
    # on a small box with smaller grains, so that it holds several seeds.
    p = workloads.fontainebleau(5, 1, n=64, grain_um=40.0)
    assert p["cd"] == pytest.approx(6 * 0.85 * 64 / (np.pi * 40.0**3))
    want = oracle.run(p)
    out, st = Q.generate(p)
    assert np.array_equal(out.cpu().numpy(), want.phase)
    assert (st.solid_count, st.steps, st.status, st.n_seeds) == \
           (want.solid_count, want.steps, want.status, want.n_accepted)


def test_largest_grid_properties(Q):
    # Close to the 2^32-voxel limit of 32-bit voxel indices, with a ragged
    # row (one pad bit per row) and a saturated face probability (the Eq. 1
    # clamp): properties the oracle need not compute at this size.
    p = dict(workloads.small_64(), nx=2047, ny=2048, nz=1024, cd=2e-6, spacing_s=0,
             g_face=0.2, g_edge=0.05, g_corner=0.0125, target_solid_fraction=0.3, seed=99)
    n = p["nx"] * p["ny"] * p["nz"]
    assert n < 2**32
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow()
        assert st.status == Q.QSGS_OK
        assert st.solid_count == st.target_count == int(np.floor(0.3 * n + 0.5))
        assert 0 < st.n_seeds <= st.n_candidates
        words = g.fetch(fmt="packed").view(p["nz"] * p["ny"], -1)
        assert words.shape[1] == 64
        assert int((words[:, -1] < 0).sum()) == 0          # the pad bit (bit 31) stays 0
        table = torch.tensor([bin(i).count("1") for i in range(256)], device=words.device)
        assert int(table[words.contiguous().view(torch.uint8).long()].sum()) == st.solid_count
    finally:
        g.close()


@pytest.mark.parametrize("dims", [(3, 3, 3), (5, 7, 4), (31, 9, 10), (32, 12, 9), (33, 10, 11),
                                  (64, 7, 6), (70, 20, 17), (95, 13, 5)])
def test_periodic_parity(oracle, Q, dims):
    # The torus (R11): x wraps inside one word, across words and at ragged
    # row ends; y and z wrap across rows and planes; spacing wraps too.
    nx, ny, nz = dims
    n = nx * ny * nz
    for s, cd in ((0, 0.02), (3, 0.05), (7, 0.08)):
        p = dict(workloads.small_64(), nx=nx, ny=ny, nz=nz, spacing_s=s, cd=cd,
                 g_face=0.05, g_edge=0.02, g_corner=0.01, target_solid_fraction=0.8,
                 seed=n + s, periodic=1)
        assert_same(oracle, Q, p)


def test_periodic_batch_and_fullfield(oracle, Q):
    rng = np.random.default_rng(77)
    params = [dict(workloads.random_small(rng, max_edge=30), periodic=1) for _ in range(5)]
    params = [dict(p, nx=max(3, p["nx"]), ny=max(3, p["ny"]), nz=max(3, p["nz"])) for p in params]
    gens = [Q.Generator(p) for p in params]
    b = Q.Batch(len(params), sum(Q.word_count(p) for p in params))
    try:
        b.set_members(gens)
        for g, st, p in zip(gens, b.run(), params):
            want = oracle.run(p)
            assert np.array_equal(g.fetch().cpu().numpy(), want.phase), p
            assert (st.solid_count, st.steps, st.front_size) == \
                   (want.solid_count, want.steps, want.front_size), p
    finally:
        b.close()
        for g in gens:
            g.close()
    p = params[0]
    g = Q.Generator(p)
    try:
        g.set_mode(Q.QSGS_MODE_FULLFIELD)
        g.seed()
        g.grow()
        assert np.array_equal(g.fetch().cpu().numpy(), oracle.run(p).phase)
    finally:
        g.close()


@pytest.mark.parametrize("periodic", [0, 1])
def test_phases_match_the_oracle(oracle, Q, periodic):
    # Independent discrete phases (R12): each grows on the cells no earlier
    # phase holds; the label maps and every phase's statistics agree.
    rng = np.random.default_rng(300 + periodic)
    for trial in range(3):
        dims = dict(nx=int(rng.integers(20, 70)), ny=int(rng.integers(12, 40)),
                    nz=int(rng.integers(10, 30)), periodic=periodic)
        phases = []
        for frac, cd, s in ((0.35, 0.004, 3), (0.2, 0.01, 0), (0.15, 0.02, 5)):
            phases.append(dict(workloads.small_64(), **dims, cd=cd, spacing_s=s,
                               g_face=0.05, g_edge=0.02, g_corner=0.01,
                               target_solid_fraction=frac, seed=int(rng.integers(0, 2**62))))
        want, results = oracle.run_phases(phases)
        labels, stats = Q.generate_phases(phases)
        assert np.array_equal(labels.cpu().numpy(), want), (trial, dims)
        for st, r in zip(stats, results):
            assert (st.solid_count, st.steps, st.status, st.n_seeds, st.front_size) == \
                   (r.solid_count, r.steps, r.status, r.n_accepted, r.front_size)


@pytest.mark.parametrize("periodic", [0, 1])
def test_interacting_phase_matches_the_oracle(oracle, Q, periodic):
    # Reading R13: the phase also grows into cells of earlier phases (random
    # label maps and interaction tables); grid and statistics agree, the
    # per-step front sums included.
    rng = np.random.default_rng(320 + periodic)
    for trial in range(5):
        p = dict(workloads.small_64(), nx=int(rng.integers(20, 70)), ny=int(rng.integers(12, 40)),
                 nz=int(rng.integers(10, 30)), periodic=periodic, cd=0.006,
                 spacing_s=int(rng.integers(0, 5)), g_face=0.06, g_edge=0.02, g_corner=0.01,
                 target_solid_fraction=float(rng.uniform(0.3, 0.7)),
                 seed=int(rng.integers(0, 2**62)), max_steps=600)
        shape = (p["nz"], p["ny"], p["nx"])
        n_labels = int(rng.integers(1, 4))
        lab = rng.integers(1, n_labels + 1, size=shape).astype(np.uint8)
        lab[rng.random(shape) >= rng.uniform(0.2, 0.6)] = 0
        inter = rng.uniform(0.0, 0.5, size=(n_labels, 3)) * (rng.random((n_labels, 3)) < 0.7)
        want = oracle.run(p, blocked=lab, inter=inter)
        g = Q.Generator(p)
        try:
            labels = torch.from_numpy(lab).cuda()
            g.set_interaction(labels, inter.tolist())
            g.seed()
            st = g.grow()
            got = g.fetch().cpu().numpy()
            assert np.array_equal(got, want.phase), (trial, p)
            assert (st.solid_count, st.steps, st.status, st.front_size, st.n_seeds) == \
                   (want.solid_count, want.steps, want.status, want.front_size, want.n_accepted)
            assert st.sum_front == int(want.log["front"].sum())
        finally:
            g.close()


def test_interacting_phases_generate_matches_the_oracle(oracle, Q):
    rng = np.random.default_rng(330)
    for periodic in (0, 1):
        dims = dict(nx=int(rng.integers(24, 60)), ny=int(rng.integers(16, 40)),
                    nz=int(rng.integers(12, 30)), periodic=periodic)
        phases = []
        for frac, cd, s in ((0.35, 0.004, 3), (0.25, 0.01, 0), (0.2, 0.02, 4)):
            phases.append(dict(workloads.small_64(), **dims, cd=cd, spacing_s=s,
                               g_face=0.05, g_edge=0.02, g_corner=0.01, max_steps=600,
                               target_solid_fraction=frac, seed=int(rng.integers(0, 2**62))))
        spec = [None, {1: (0.3, 0.1, 0.05)}, {1: (0.2, 0.0, 0.0), 2: (0.0, 0.25, 0.3)}]
        want, results = oracle.run_phases(phases, spec)
        labels, stats = Q.generate_phases(phases, interactions=spec)
        assert np.array_equal(labels.cpu().numpy(), want), periodic
        for st, r in zip(stats, results):
            assert (st.solid_count, st.steps, st.status, st.n_seeds, st.front_size) == \
                   (r.solid_count, r.steps, r.status, r.n_accepted, r.front_size)


def test_interaction_is_single_path_lists_only(Q):
    p = dict(workloads.small_64(), nx=20, ny=20, nz=20)
    g = Q.Generator(p)
    b = Q.Batch(1, Q.word_count(p))
    try:
        labels = torch.zeros((20, 20, 20), dtype=torch.uint8, device="cuda")
        labels[:, :, :5] = 1
        g.set_interaction(labels, [(0.5, 0.5, 0.5)])
        with pytest.raises(Q.QsgsError):
            g.set_mode(Q.QSGS_MODE_FULLFIELD)
        with pytest.raises(Q.QsgsError):
            b.set_members([g])
        g.set_interaction(None, None)       # cleared: both allowed again
        b.set_members([g])
        g.set_mode(Q.QSGS_MODE_FULLFIELD)
    finally:
        b.close()
        g.close()


def test_blocked_single_phase_and_batch(oracle, Q):
    rng = np.random.default_rng(310)
    params = [dict(workloads.random_small(rng, max_edge=26), cd=0.03, max_steps=0)
              for _ in range(4)]
    blocks, gens = [], []
    for p in params:
        shape = (p["nz"], p["ny"], p["nx"])
        blk = rng.random(shape) < 0.3
        words = ((p["nx"] + 31) // 32)
        packed = np.zeros((p["nz"], p["ny"], words * 32), dtype=bool)
        packed[:, :, :p["nx"]] = blk
        w32 = np.packbits(packed, axis=-1, bitorder="little").view(np.uint32).reshape(-1)
        t = torch.from_numpy(w32.view(np.int32).copy()).cuda()
        g = Q.Generator(p)
        g.set_blocked(t)
        blocks.append((blk, t))
        gens.append(g)
    b = Q.Batch(len(params), sum(Q.word_count(p) for p in params))
    try:
        b.set_members(gens[:2])
        stats = b.run()
        for g, st, p, (blk, _) in zip(gens[:2], stats, params, blocks):
            want = oracle.run(p, blocked=blk)
            assert np.array_equal(g.fetch().cpu().numpy(), want.phase)
            assert st.solid_count == want.solid_count and st.steps == want.steps
        for g, p, (blk, _) in zip(gens[2:], params[2:], blocks[2:]):
            g.seed()
            st = g.grow()
            want = oracle.run(p, blocked=blk)
            assert np.array_equal(g.fetch().cpu().numpy(), want.phase)
            assert (st.solid_count, st.front_size) == (want.solid_count, want.front_size)
    finally:
        b.close()
        for g in gens:
            g.close()


def test_bounded_wait_gives_up_and_the_handle_recovers(Q):
    # Failure detection without a fault: with a two-poll limit the look-back
    # waits of the order-preserving passes give up (their predecessors have
    # not published yet), the kernels finish, and the host reads
    # QSGS_ERR_TIMEOUT; the same handle with the default limit then gives
    # the golden realization.
    row = _golden("single_400")[0]
    g = Q.Generator(row["params"])
    try:
        Q.qsgs_set_spin_limit(g.handle, 2)
        codes = []
        for _ in range(8):
            g.seed()
            try:
                g.grow()
                codes.append(Q.QSGS_OK)
            except Q.QsgsError as e:
                codes.append(e.code)
                break
        assert codes[-1] == Q.QSGS_ERR_TIMEOUT, codes
        Q.qsgs_set_spin_limit(g.handle, 0)
        g.seed()
        st = g.grow()
        phase = g.fetch().cpu().numpy()
        assert hashlib.sha256(phase.tobytes()).hexdigest() == row["sha256_u8"]
        assert (st.solid_count, st.steps, st.status) == (row["solid_count"], row["steps"],
                                                         row["status"])
    finally:
        g.close()
