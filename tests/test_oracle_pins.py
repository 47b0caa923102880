"""Pins of the CPU oracle to things other than itself.

Each test checks the oracle against what the paper or mathematics fixes:
an independent Philox implementation, exact rational evaluation of Eq. 1,
binomial statistics of the Bernoulli draws, closed forms of the growth at
probability 0 or 1 (dilations computed by scipy), brute-force spacing and
front checks, and the equivalence of Algorithm 3 with Algorithm 2.
"""
import itertools
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

from paper_2602_11734_gb300 import workloads

TWO32 = 2**32


# --------------------------------------------------------------------------
# Philox4x32-10 against torch's header-only engine (an independent
# implementation of Salmon et al.'s generator), compiled and run here.
# --------------------------------------------------------------------------
_HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdint>
#include <cstdio>
int main() {
  unsigned c0, c1, c2, c3, k0, k1;
  while (std::scanf("%x %x %x %x %x %x", &c0, &c1, &c2, &c3, &k0, &k1) == 6) {
    uint64_t seed = (uint64_t)k1 << 32 | k0;
    at::Philox4_32 e(seed, (uint64_t)c3 << 32 | c2, 0);
    e.set_offset((uint64_t)c1 << 32 | c0);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%08x %08x %08x %08x\n", a, b, c, d);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("torch Philox header not available")
    d = tmp_path_factory.mktemp("philox")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(_HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)

    def run(rows):
        text = "".join(" ".join(f"{v:08x}" for v in r) + "\n" for r in rows)
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True)
        return [tuple(int(w, 16) for w in line.split()) for line in out.stdout.splitlines()]

    return run


def test_philox_matches_torch_engine(oracle, torch_philox):
    rng = np.random.default_rng(11)
    rows = [tuple(int(v) for v in rng.integers(0, TWO32, size=6, dtype=np.uint64)) for _ in range(2000)]
    rows += [(0, 0, 0, 0, 0, 0), (0xFFFFFFFF,) * 6, (1, 0, 0xFFFFFFFF, 0x100, 1, 0),
             (123, 0, 7, 0x205, 0xDEADBEEF, 0x12345678)]
    ref = torch_philox(rows)
    for r, want in zip(rows, ref):
        got = tuple(int(v) for v in oracle.philox(r[:4], r[4:]))
        assert got == want, (r, got, want)


def test_philox_key_and_counter_sensitivity(oracle):
    # Every input word changes the block (a dropped word would not).
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for i in range(6):
        w = [1, 2, 3, 4, 5, 6]
        w[i] ^= 1
        assert not np.array_equal(oracle.philox(w[:4], w[4:]), base)


# --------------------------------------------------------------------------
# Directions
# --------------------------------------------------------------------------
def test_directions_are_the_26_neighbours(oracle):
    dirs, cls = oracle.directions()
    as_set = {tuple(int(v) for v in d) for d in dirs}
    assert as_set == {d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)}
    assert len(as_set) == 26
    nonzero = (dirs != 0).sum(axis=1)
    assert np.array_equal(cls, nonzero - 1)
    assert list(cls) == [0] * 6 + [1] * 12 + [2] * 8
    for c in range(3):  # within a class: lexicographic in (dz, dy, dx)
        keys = [(d[2], d[1], d[0]) for d in dirs[cls == c]]
        assert keys == sorted(keys)


# --------------------------------------------------------------------------
# Parameters and Eq. 1
# --------------------------------------------------------------------------
def test_targets_of_the_workloads(oracle):
    nt, ts, tr = oracle.targets(workloads.small_64())
    assert nt == 183501                    # 0.70 * 262144 = 183500.8
    assert ts == 8589934                   # floor(0.002 * 2^32)
    assert tr == (42949672, 10737418, 2684354)
    assert oracle.targets(workloads.single_400())[0] == 51_200_000
    sweep = [oracle.targets(p)[0] for p in workloads.sweep_500()[::5]]
    assert sweep == [115_000_000, 110_000_000, 105_000_000, 100_000_000, 93_750_000]


@pytest.mark.parametrize("bad", [dict(nx=0), dict(cd=1.5), dict(cd=-0.1), dict(g_face=2.0),
                                 dict(g_corner=float("nan")), dict(target_count=10**6),
                                 dict(target_solid_fraction=1.2),
                                 dict(nx=2**11, ny=2**11, nz=2**10)])
def test_targets_reject_invalid(oracle, bad):
    p = dict(nx=8, ny=8, nz=8, target_solid_fraction=0.5)
    p.update(bad)
    with pytest.raises(ValueError):
        oracle.targets(p)


def _eq1_paper(g_ref_t, nt, n, c):
    """The paper's Eq. 1 as printed, in exact rationals:
    G = G_ref (phi_s - 0.95 phi_a) / (0.05 phi_s)."""
    phi_s, phi_a = Fraction(nt, n), Fraction(c, n)
    g = Fraction(g_ref_t) * (phi_s - Fraction(95, 100) * phi_a) / (Fraction(5, 100) * phi_s)
    return min(TWO32, g.numerator // g.denominator)


def test_eq1_threshold_matches_exact_rational_form(oracle):
    rng = np.random.default_rng(5)
    for _ in range(3000):
        n = int(rng.integers(1, 2**32))
        nt = int(rng.integers(1, n + 1))
        c = int(rng.integers(0, nt + 1))
        t_ref = int(rng.integers(0, TWO32 + 1))
        assert oracle.threshold(t_ref, nt, c) == _eq1_paper(t_ref, nt, n, c)


def test_eq1_endpoints(oracle):
    # G(0) = 20 G_ref and G(phi_s) = G_ref, by Eq. 1.
    for t_ref in (0, 1, 2684354, 42949672, 2**31, TWO32):
        for nt in (1, 7, 183501, 51_200_000):
            assert oracle.threshold(t_ref, nt, 0) == min(TWO32, 20 * t_ref)
            assert oracle.threshold(t_ref, nt, nt) == t_ref
    # non-increasing in c
    vals = [oracle.threshold(42949672, 1000, c) for c in range(0, 1001, 10)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))


# --------------------------------------------------------------------------
# Bernoulli seeding (Sec. 2.1 step 2)
# --------------------------------------------------------------------------
def test_seeding_count_is_binomial(oracle):
    p = dict(nx=32, ny=32, nz=32, cd=0.01, target_solid_fraction=0.5)
    t_seed = oracle.targets(p)[1]
    prob = t_seed / TWO32
    total, trials = 0, 0
    for s in range(200):
        c = oracle.seed_candidates(dict(p, seed=s))
        assert np.all(np.diff(c.astype(np.int64)) > 0) and (c.size == 0 or c[-1] < 32**3)
        total += c.size
        trials += 32**3
    z = (total - trials * prob) / np.sqrt(trials * prob * (1 - prob))
    assert abs(z) < 5, z


def test_seeding_draws_are_independent_within_a_philox_block(oracle):
    # Voxels 4g..4g+3 share one Philox block but use different words: the
    # number of candidates per block must follow Binomial(4, p).
    p = dict(nx=64, ny=64, nz=16, cd=0.3, target_solid_fraction=0.5)
    prob = oracle.targets(p)[1] / TWO32
    hist = np.zeros(5)
    for s in range(6):
        c = oracle.seed_candidates(dict(p, seed=s))
        per_group = np.bincount(c // 4, minlength=64 * 64 * 16 // 4)
        hist += np.bincount(per_group, minlength=5)
    from scipy import stats
    expect = np.array([stats.binom.pmf(k, 4, prob) for k in range(5)]) * hist.sum()
    chi2 = ((hist - expect) ** 2 / expect).sum()
    assert chi2 < 30, (hist, expect)


def test_seeding_extremes(oracle):
    p = dict(nx=5, ny=3, nz=7, target_solid_fraction=0.5, seed=9)
    assert oracle.seed_candidates(dict(p, cd=0.0)).size == 0
    assert np.array_equal(oracle.seed_candidates(dict(p, cd=1.0)), np.arange(105))


# --------------------------------------------------------------------------
# Seed spacing (Sec. 2.3, Fig. 1 D): brute force and scipy dilation
# --------------------------------------------------------------------------
def _l1(a, b, dims):
    nx, ny, _ = dims
    ax, ay, az = a % nx, (a // nx) % ny, a // (nx * ny)
    bx, by, bz = b % nx, (b // nx) % ny, b // (nx * ny)
    return abs(int(ax) - int(bx)) + abs(int(ay) - int(by)) + abs(int(az) - int(bz))


def _spacing_by_dilation(cand, dims, s):
    nx, ny, nz = dims
    mask = np.zeros((nz, ny, nx), dtype=bool)
    struct = ndimage.generate_binary_structure(3, 1)
    acc = []
    for v in cand:
        z, y, x = v // (nx * ny), (v // nx) % ny, v % nx
        if s > 1 and mask[z, y, x]:
            acc.append(False)
            continue
        acc.append(True)
        if s > 1:
            pt = np.zeros_like(mask)
            pt[z, y, x] = True
            mask |= ndimage.binary_dilation(pt, structure=struct, iterations=s - 1) if s > 2 \
                else ndimage.binary_dilation(pt, structure=struct)
    return np.array(acc, dtype=bool)


@pytest.mark.parametrize("s", [0, 1, 2, 3, 4, 6, 9])
def test_spacing_is_greedy_maximal_and_separated(oracle, s):
    rng = np.random.default_rng(100 + s)
    for trial in range(6):
        dims = tuple(int(v) for v in rng.integers(3, 17, size=3))
        n = dims[0] * dims[1] * dims[2]
        p = dict(nx=dims[0], ny=dims[1], nz=dims[2], spacing_s=s, cd=0.05,
                 target_solid_fraction=0.5, seed=int(rng.integers(0, 2**32)))
        cand = oracle.seed_candidates(p)
        if cand.size == 0:
            cand = np.sort(rng.choice(n, size=min(n, 10), replace=False)).astype(np.uint32)
        acc = oracle.spacing(p, cand)
        kept = cand[acc]
        for i, j in itertools.combinations(range(kept.size), 2):
            assert _l1(kept[i], kept[j], dims) >= s
        for i in np.nonzero(~acc)[0]:
            assert any(_l1(cand[i], k, dims) < s for k in kept if k < cand[i])
        assert np.array_equal(acc, _spacing_by_dilation(cand, dims, s))


# --------------------------------------------------------------------------
# Active front (Sec. 2.3 step 2)
# --------------------------------------------------------------------------
def _front_bruteforce(phase):
    solid = phase.astype(bool)
    void_near = ndimage.binary_dilation(~solid, structure=np.ones((3, 3, 3), bool))
    return np.flatnonzero(solid & void_near)


def test_front_matches_bruteforce(oracle):
    rng = np.random.default_rng(3)
    for _ in range(30):
        nx, ny, nz = (int(v) for v in rng.integers(1, 14, size=3))
        phase = (rng.random((nz, ny, nx)) < rng.uniform(0.1, 0.99)).astype(np.uint8)
        got = oracle.front(dict(nx=nx, ny=ny, nz=nz, target_solid_fraction=0.5), phase)
        assert np.array_equal(got, _front_bruteforce(phase))


# --------------------------------------------------------------------------
# Growth: closed forms at probability 0 and 1 (Algorithm 3 semantics)
# --------------------------------------------------------------------------
def _seeds_phase(oracle, p):
    cand = oracle.seed_candidates(p)
    acc = oracle.spacing(p, cand)
    ph = np.zeros(p["nx"] * p["ny"] * p["nz"], dtype=bool)
    ph[cand[acc]] = True
    return ph.reshape(p["nz"], p["ny"], p["nx"])


def _structure(classes):
    st = np.zeros((3, 3, 3), dtype=bool)
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        k = abs(dx) + abs(dy) + abs(dz)
        if k == 0 or (k - 1) in classes:
            st[dz + 1, dy + 1, dx + 1] = True
    return st


def _dilate(seeds, classes, k):
    out = seeds.copy()
    st = _structure(classes)
    for _ in range(k):
        out = ndimage.binary_dilation(out, structure=st)
    return out


@pytest.mark.parametrize("classes", [(0, 1, 2), (0,), (1,), (2,), (0, 2)])
def test_unit_probability_growth_is_a_dilation(oracle, classes):
    g = [1.0 if c in classes else 0.0 for c in range(3)]
    rng = np.random.default_rng(7)
    for trial in range(4):
        nx, ny, nz = (int(v) for v in rng.integers(4, 15, size=3))
        n = nx * ny * nz
        k = int(rng.integers(1, 5))
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.01, g_face=g[0], g_edge=g[1], g_corner=g[2],
                 spacing_s=int(rng.integers(0, 4)), target_count=n, seed=trial, max_steps=k)
        seeds = _seeds_phase(oracle, p)
        if not seeds.any():
            continue
        r = oracle.run(p)
        want = seeds.copy()
        steps = 0
        for _ in range(k):
            nxt = _dilate(want, classes, 1)
            if np.array_equal(nxt, want):
                break
            want, steps = nxt, steps + 1
        assert np.array_equal(r.phase.astype(bool), want)
        assert r.solid_count == int(want.sum())
        assert r.steps == steps
        full = want.all()
        exp_status = oracle.DONE if full else (oracle.MAX_STEPS if steps == k else oracle.STALLED)
        assert r.status == exp_status


def test_zero_probability_stalls_with_seeds_only(oracle):
    p = dict(nx=12, ny=9, nz=10, cd=0.02, target_solid_fraction=0.8, seed=4)
    r = oracle.run(p)
    assert r.status == oracle.STALLED and r.steps == 0
    assert np.array_equal(r.phase.astype(bool), _seeds_phase(oracle, p))


def test_edge_only_growth_stalls_on_its_sublattice(oracle):
    # Edge moves keep x+y+z mod 2; growth stops once a parity class is full.
    p = dict(nx=6, ny=6, nz=6, cd=0.0, g_edge=1.0, target_solid_fraction=0.9, seed=1)
    p["cd"] = 1.0 / 216
    for seed in range(20):
        q = dict(p, seed=seed)
        seeds = _seeds_phase(oracle, q)
        if seeds.sum() != 1:
            continue
        r = oracle.run(q)
        assert r.status == oracle.STALLED
        z, y, x = np.nonzero(seeds)
        par = (x[0] + y[0] + z[0]) % 2
        zz, yy, xx = np.indices((6, 6, 6))
        assert np.array_equal(r.phase.astype(bool), (xx + yy + zz) % 2 == par)
        return
    pytest.skip("no single-seed realization found")


def test_exact_target_trim_keeps_lowest_indices(oracle):
    # At probability 1 the step-k claims are D_k \ D_{k-1}; the trim keeps
    # the lowest indices among them so that exactly Nt voxels are solid.
    rng = np.random.default_rng(21)
    checked = 0
    for trial in range(40):
        nx, ny, nz = (int(v) for v in rng.integers(5, 13, size=3))
        n = nx * ny * nz
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.01, g_face=1.0, g_edge=1.0, g_corner=1.0, seed=trial)
        seeds = _seeds_phase(oracle, p)
        if not seeds.any() or seeds.all():
            continue
        d = [seeds]
        while not d[-1].all():
            d.append(_dilate(d[-1], (0, 1, 2), 1))
        k = int(rng.integers(1, len(d)))
        lo, hi = int(d[k - 1].sum()), int(d[k].sum())
        if hi - lo < 2:
            continue
        nt = int(rng.integers(lo + 1, hi))
        r = oracle.run(dict(p, target_count=nt))
        claimed = np.flatnonzero((d[k] & ~d[k - 1]).ravel())
        want = d[k - 1].ravel().copy()
        want[claimed[: nt - lo]] = True
        assert r.status == oracle.DONE and r.steps == k and r.solid_count == nt
        assert np.array_equal(r.phase.ravel().astype(bool), want)
        checked += 1
    assert checked >= 10


def test_seed_cap_keeps_lowest_seeds(oracle):
    p = dict(nx=10, ny=10, nz=10, cd=0.2, g_face=0.3, seed=2)
    seeds = np.flatnonzero(_seeds_phase(oracle, p).ravel())
    assert seeds.size > 20
    r = oracle.run(dict(p, target_count=17))
    assert r.status == oracle.DONE and r.steps == 0 and r.solid_count == 17
    assert np.array_equal(np.flatnonzero(r.phase.ravel()), seeds[:17])


# --------------------------------------------------------------------------
# Single-attempt probabilities per class (Eq. 1 at c_0, R2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cls,s", [(0, 3), (1, 5), (2, 7)])
def test_first_step_claim_rate_per_class(oracle, cls, s):
    # Seeds at L1 >= s have disjoint class-neighbourhoods, so the step-0
    # claims are independent Bernoulli trials with p = T_cls(c_0) / 2^32.
    g = [0.0, 0.0, 0.0]
    g[cls] = 0.02
    dirs, dcls = oracle.directions()
    offs = dirs[dcls == cls]
    n_edge = 20
    hits = trials = 0
    psum = 0.0
    for seed in range(150):
        p = dict(nx=n_edge, ny=n_edge, nz=n_edge, cd=0.004, g_face=g[0], g_edge=g[1],
                 g_corner=g[2], spacing_s=s, target_solid_fraction=0.9, seed=seed)
        seeds = _seeds_phase(oracle, p)
        z, y, x = np.nonzero(seeds)
        m = 0
        for o in offs:
            xx, yy, zz = x + o[0], y + o[1], z + o[2]
            m += int(((xx >= 0) & (xx < n_edge) & (yy >= 0) & (yy < n_edge) &
                      (zz >= 0) & (zz < n_edge)).sum())
        if m == 0:
            continue
        r = oracle.run(dict(p, max_steps=1))
        nt = oracle.targets(p)[0]
        t_ref = oracle.targets(p)[2][cls]
        prob = _eq1_paper(t_ref, nt, n_edge**3, int(seeds.sum())) / TWO32
        hits += int(r.log[0]["claimed"])
        trials += m
        psum += m * prob
    mean_p = psum / trials
    z = (hits - psum) / np.sqrt(trials * mean_p * (1 - mean_p))
    assert abs(z) < 5, (hits, psum, trials)


# --------------------------------------------------------------------------
# Algorithm 3 == Algorithm 2 (Sec. 2.3: same growth statistics), invariants
# --------------------------------------------------------------------------
def test_list_indexed_equals_full_field(oracle):
    rng = np.random.default_rng(2024)
    for _ in range(60):
        p = workloads.random_small(rng, max_edge=12)
        a = oracle.run(p)
        b = oracle.run_fullfield(p)
        assert np.array_equal(a.phase, b.phase), p
        assert (a.solid_count, a.steps, a.status, a.front_size) == \
               (b.solid_count, b.steps, b.status, b.front_size), p


def test_run_invariants(oracle):
    rng = np.random.default_rng(77)
    cases = [workloads.random_small(rng, max_edge=18) for _ in range(25)]
    cases.append(dict(workloads.small_64(), nx=24, ny=20, nz=22))
    for p in cases:
        r = oracle.run(p)
        nt, _, t_ref = oracle.targets(p)
        assert int(r.phase.sum()) == r.solid_count
        if r.status == oracle.DONE:
            assert r.solid_count == nt
        else:
            assert r.solid_count < nt
        assert r.front_size == _front_bruteforce(r.phase).size
        log = r.log
        assert log.size == r.steps
        if log.size:
            assert np.all(np.diff(log["solid_before"].astype(np.int64)) >= 0)
            assert np.array_equal(log["t"], np.arange(log.size))
            for row in log[:5]:
                n = p["nx"] * p["ny"] * p["nz"]
                for k in range(3):
                    assert int(row["thr"][k]) == _eq1_paper(t_ref[k], nt, n, int(row["solid_before"]))
        if r.steps and r.status == oracle.DONE:
            last = log[-1]
            assert int(last["solid_before"]) + min(int(last["claimed"]),
                                                   nt - int(last["solid_before"])) == nt


def test_growth_draws_within_a_block_are_independent(oracle):
    # Directions 0..3 share one Philox block and use different words: the
    # joint success of two of them must have probability p^2 (the same word
    # reused would give p).  Isolated seeds, faces only, one step.
    dirs, _ = oracle.directions()
    n_edge = 20
    both = single = m = 0
    prob = None
    for seed in range(120):
        p = dict(nx=n_edge, ny=n_edge, nz=n_edge, cd=0.004, g_face=0.02, spacing_s=3,
                 target_solid_fraction=0.9, seed=seed)
        seeds = _seeds_phase(oracle, p)
        r = oracle.run(dict(p, max_steps=1))
        nt, _, t_ref = oracle.targets(p)
        prob = _eq1_paper(t_ref[0], nt, n_edge**3, int(seeds.sum())) / TWO32
        ph = r.phase.astype(bool)
        for z, y, x in zip(*np.nonzero(seeds)):
            hit = []
            for d in (0, 1):
                xx, yy, zz = x + dirs[d][0], y + dirs[d][1], z + dirs[d][2]
                if not (0 <= xx < n_edge and 0 <= yy < n_edge and 0 <= zz < n_edge):
                    break
                hit.append(bool(ph[zz, yy, xx]))
            if len(hit) < 2:
                continue
            m += 1
            single += hit[0]
            both += hit[0] and hit[1]
    exp = m * prob * prob
    z = (both - exp) / np.sqrt(m * prob * prob * (1 - prob * prob))
    assert abs(z) < 5, (both, exp, single, m)


# --------------------------------------------------------------------------
# R1 counter layout, evaluated with the independent engine
# --------------------------------------------------------------------------
def test_seeding_counter_layout(oracle, torch_philox):
    p = dict(nx=13, ny=7, nz=5, cd=0.2, target_solid_fraction=0.5, seed=0x1234567890ABCDEF)
    t_seed = oracle.targets(p)[1]
    n = 13 * 7 * 5
    k0, k1 = p["seed"] & 0xFFFFFFFF, p["seed"] >> 32
    rows = [((g & 0xFFFFFFFF), g >> 32, 0xFFFFFFFF, 0x100, k0, k1) for g in range((n + 3) // 4)]
    blocks = torch_philox(rows)
    want = [v for v in range(n) if blocks[v >> 2][v & 3] < t_seed]
    assert list(oracle.seed_candidates(p)) == want


def _growth_step_by_layout(seeds, shape, p, thr, torch_philox, dirs, cls):
    """One growth step from `seeds`, restated from R1: the targets of a
    source are its in-domain neighbours that are void at the start of the
    step (with a positive class threshold); the r-th target of class k (in
    the canonical direction order) draws word r & 3 of the Philox block
    (a, 0, t = 0, 0x200 | B_k + r >> 2), B = (0, 2, 5); a target is claimed
    when some draw is below its class threshold."""
    nz, ny, nx = shape
    k0, k1 = p["seed"] & 0xFFFFFFFF, p["seed"] >> 32
    first = (0, 2, 5)
    want = seeds.copy()
    for a in np.flatnonzero(seeds.ravel()):
        z, y, x = a // (nx * ny), (a // nx) % ny, a % nx
        blocks = torch_philox([(int(a), 0, 0, 0x200 | b, k0, k1) for b in range(7)])
        rank = [0, 0, 0]
        for d in range(26):
            xx, yy, zz = x + dirs[d][0], y + dirs[d][1], z + dirs[d][2]
            if not (0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz) or seeds[zz, yy, xx]:
                continue
            k = cls[d]
            if thr[k] == 0:
                continue
            r = rank[k]
            rank[k] += 1
            if blocks[first[k] + (r >> 2)][r & 3] < thr[k]:
                want[zz, yy, xx] = True
    return want


def test_growth_counter_layout(oracle, torch_philox):
    # One step from isolated seeds (every interior neighbour a target) and
    # from touching seeds (solid neighbours shift the ranks): the claimed set
    # is exactly the one the R1 layout gives with the independent engine.
    dirs, cls = oracle.directions()
    checked = 0
    for seed in range(40):
        for spacing, cd in ((7, 0.003), (0, 0.06)):
            p = dict(nx=16, ny=15, nz=14, cd=cd, g_face=0.03, g_edge=0.02, g_corner=0.01,
                     spacing_s=spacing, target_solid_fraction=0.9,
                     seed=seed * 0x9E3779B97F4A7C15 % 2**64)
            seeds = _seeds_phase(oracle, p)
            if not seeds.any():
                continue
            nt, _, t_ref = oracle.targets(p)
            thr = [oracle.threshold(t_ref[k], nt, int(seeds.sum())) for k in range(3)]
            want = _growth_step_by_layout(seeds, (14, 15, 16), p, thr, torch_philox, dirs, cls)
            r = oracle.run(dict(p, max_steps=1))
            assert np.array_equal(r.phase.astype(bool), want)
            checked += 1
    assert checked > 50


def test_growth_layout_skips_dead_classes(oracle, torch_philox):
    # A class with a zero threshold has no targets: the ranks of the live
    # classes do not count its directions (edges only here).
    dirs, cls = oracle.directions()
    checked = 0
    for seed in range(20):
        p = dict(nx=12, ny=13, nz=11, cd=0.05, g_face=0.0, g_edge=0.3, g_corner=0.0,
                 spacing_s=0, target_solid_fraction=0.95, seed=7 + seed)
        seeds = _seeds_phase(oracle, p)
        if not seeds.any():
            continue
        nt, _, t_ref = oracle.targets(p)
        thr = [oracle.threshold(t_ref[k], nt, int(seeds.sum())) for k in range(3)]
        assert thr[0] == 0 and thr[2] == 0 and thr[1] > 0
        want = _growth_step_by_layout(seeds, (11, 13, 12), p, thr, torch_philox, dirs, cls)
        r = oracle.run(dict(p, max_steps=1))
        assert np.array_equal(r.phase.astype(bool), want)
        checked += 1
    assert checked > 10


# --------------------------------------------------------------------------
# Periodic option (R11): the torus of the roll in Sec. 2.2 / Algorithm 2
# --------------------------------------------------------------------------
_OFFSETS = [(dz, dy, dx) for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3)
            if (dz, dy, dx) != (0, 0, 0)]


def _torus_l1(a, b, dims):
    nx, ny, nz = dims
    (xa, ya, za), (xb, yb, zb) = ((v % nx, (v // nx) % ny, v // (nx * ny)) for v in (int(a), int(b)))
    d = 0
    for u, w, m in ((xa, xb, nx), (ya, yb, ny), (za, zb, nz)):
        k = abs(u - w)
        d += min(k, m - k)
    return d


def test_periodic_front_matches_roll_bruteforce(oracle):
    rng = np.random.default_rng(31)
    for _ in range(25):
        nx, ny, nz = (int(v) for v in rng.integers(3, 12, size=3))
        phase = rng.random((nz, ny, nx)) < rng.uniform(0.2, 0.99)
        void_near = np.zeros_like(phase)
        for dz, dy, dx in _OFFSETS:
            void_near |= np.roll(~phase, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        got = oracle.front(dict(nx=nx, ny=ny, nz=nz, target_solid_fraction=0.5, periodic=1),
                           phase.astype(np.uint8))
        assert np.array_equal(got, np.flatnonzero(phase & void_near))


@pytest.mark.parametrize("classes", [(0, 1, 2), (0,), (2,)])
def test_periodic_unit_probability_growth_is_a_rolled_dilation(oracle, classes):
    # G = 1 on the torus: after k steps the solid set is the seeds dilated k
    # times by the class offsets, with np.roll (periodic) shifts.
    g = [1.0 if c in classes else 0.0 for c in range(3)]
    rng = np.random.default_rng(8)
    for trial in range(4):
        nx, ny, nz = (int(v) for v in rng.integers(3, 13, size=3))
        n = nx * ny * nz
        k = int(rng.integers(1, 4))
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.01, g_face=g[0], g_edge=g[1], g_corner=g[2],
                 spacing_s=int(rng.integers(0, 4)), target_count=n, seed=trial, max_steps=k,
                 periodic=1)
        seeds = _seeds_phase(oracle, p)
        if not seeds.any():
            continue
        offs = [o for o in _OFFSETS if (abs(o[0]) + abs(o[1]) + abs(o[2]) - 1) in classes]
        want = seeds.copy()
        for _ in range(k):
            nxt = want.copy()
            for o in offs:
                nxt |= np.roll(want, shift=o, axis=(0, 1, 2))
            if np.array_equal(nxt, want):
                break
            want = nxt
        r = oracle.run(p)
        assert np.array_equal(r.phase.astype(bool), want)


@pytest.mark.parametrize("s", [2, 3, 5, 8])
def test_periodic_spacing_uses_the_torus_distance(oracle, s):
    rng = np.random.default_rng(200 + s)
    for trial in range(5):
        dims = tuple(int(v) for v in rng.integers(3, 15, size=3))
        p = dict(nx=dims[0], ny=dims[1], nz=dims[2], spacing_s=s, cd=0.06,
                 target_solid_fraction=0.5, seed=int(rng.integers(0, 2**32)), periodic=1)
        cand = oracle.seed_candidates(p)
        acc = oracle.spacing(p, cand)
        kept = cand[acc]
        for i, j in itertools.combinations(range(kept.size), 2):
            assert _torus_l1(kept[i], kept[j], dims) >= s
        for i in np.nonzero(~acc)[0]:
            assert any(_torus_l1(cand[i], k, dims) < s for k in kept if k < cand[i])


def test_periodic_list_indexed_equals_full_field(oracle):
    rng = np.random.default_rng(12)
    for _ in range(20):
        p = dict(nx=int(rng.integers(3, 14)), ny=int(rng.integers(3, 14)),
                 nz=int(rng.integers(3, 14)), cd=float(rng.uniform(0.002, 0.05)),
                 g_face=float(rng.uniform(0, 0.3)), g_edge=float(rng.uniform(0, 0.2)),
                 g_corner=float(rng.uniform(0, 0.1)), spacing_s=int(rng.integers(0, 5)),
                 target_solid_fraction=float(rng.uniform(0.2, 0.95)),
                 seed=int(rng.integers(0, 2**63)), periodic=1)
        a, b = oracle.run(p), oracle.run_fullfield(p)
        assert np.array_equal(a.phase, b.phase)
        assert (a.solid_count, a.steps, a.status, a.front_size) == \
               (b.solid_count, b.steps, b.status, b.front_size)


def test_periodic_needs_three_cells_per_axis(oracle):
    for dims in ((2, 5, 5), (5, 1, 5), (5, 5, 2)):
        p = dict(nx=dims[0], ny=dims[1], nz=dims[2], target_solid_fraction=0.5, periodic=1)
        with pytest.raises(Exception):
            oracle.run(p)
    oracle.run(dict(nx=3, ny=3, nz=3, target_solid_fraction=0.5, periodic=1, cd=0.2))


def test_periodic_equals_open_domain_away_from_the_faces(oracle):
    # Draws depend on (seed, voxel, step, direction) only, so a run whose
    # growth never reaches a face is the same on the torus.
    rng = np.random.default_rng(40)
    checked = 0
    for trial in range(60):
        p = dict(nx=17, ny=15, nz=16, cd=0.0008, g_face=0.3, g_edge=0.1, g_corner=0.05,
                 target_count=3000, max_steps=2, seed=trial)
        seeds = _seeds_phase(oracle, p)
        zz, yy, xx = np.nonzero(seeds)
        if len(xx) == 0 or min(xx.min(), yy.min(), zz.min()) < 3 or \
                xx.max() > 13 or yy.max() > 11 or zz.max() > 12:
            continue
        a, b = oracle.run(p), oracle.run(dict(p, periodic=1))
        assert np.array_equal(a.phase, b.phase)
        checked += 1
    assert checked >= 3


# --------------------------------------------------------------------------
# Later growing phases (R12): cells of earlier phases are blocked
# --------------------------------------------------------------------------
def _random_case(rng, periodic=0):
    lo = 3 if periodic else 2
    return dict(nx=int(rng.integers(lo, 13)), ny=int(rng.integers(lo, 13)),
                nz=int(rng.integers(lo, 13)), cd=float(rng.uniform(0.01, 0.08)),
                g_face=float(rng.uniform(0.05, 0.4)), g_edge=float(rng.uniform(0.0, 0.2)),
                g_corner=float(rng.uniform(0.0, 0.1)), spacing_s=int(rng.integers(0, 4)),
                target_solid_fraction=float(rng.uniform(0.1, 0.5)),
                seed=int(rng.integers(0, 2**63)), periodic=periodic)


def test_blocked_nothing_changes_nothing(oracle):
    rng = np.random.default_rng(51)
    for _ in range(10):
        p = _random_case(rng)
        none = np.zeros((p["nz"], p["ny"], p["nx"]), np.uint8)
        a, b = oracle.run(p), oracle.run(p, blocked=none)
        assert np.array_equal(a.phase, b.phase) and a.steps == b.steps


def test_blocked_seeding_is_the_filtered_draw(oracle):
    rng = np.random.default_rng(52)
    for _ in range(10):
        p = _random_case(rng)
        blocked = rng.random((p["nz"], p["ny"], p["nx"])) < 0.4
        free = oracle.seed_candidates(p)
        got = oracle.seed_candidates(p, blocked=blocked)
        assert np.array_equal(got, free[~blocked.reshape(-1)[free]])


def test_blocked_front_matches_bruteforce(oracle):
    rng = np.random.default_rng(53)
    for _ in range(20):
        nx, ny, nz = (int(v) for v in rng.integers(2, 12, size=3))
        blocked = rng.random((nz, ny, nx)) < 0.3
        phase = (rng.random((nz, ny, nx)) < 0.5) & ~blocked
        open_void = ~phase & ~blocked
        near = ndimage.binary_dilation(open_void, structure=np.ones((3, 3, 3), bool))
        got = oracle.front(dict(nx=nx, ny=ny, nz=nz, target_solid_fraction=0.5),
                           phase.astype(np.uint8), blocked=blocked)
        assert np.array_equal(got, np.flatnonzero(phase & near))


def test_blocked_unit_growth_is_a_geodesic_dilation(oracle):
    # G = 1: after k steps the phase is the seeds dilated k times inside the
    # unblocked cells only.
    rng = np.random.default_rng(54)
    checked = 0
    for trial in range(12):
        nx, ny, nz = (int(v) for v in rng.integers(5, 14, size=3))
        n = nx * ny * nz
        k = int(rng.integers(1, 4))
        blocked = rng.random((nz, ny, nx)) < 0.35
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.03, g_face=1.0, g_edge=1.0, g_corner=1.0,
                 target_count=n, seed=trial, max_steps=k)
        cand = oracle.seed_candidates(p, blocked=blocked)
        if cand.size == 0:
            continue
        want = np.zeros(n, bool)
        want[cand] = True
        want = want.reshape(nz, ny, nx)
        for _ in range(k):
            want = ndimage.binary_dilation(want, structure=np.ones((3, 3, 3), bool)) & ~blocked
        r = oracle.run(p, blocked=blocked)
        assert np.array_equal(r.phase.astype(bool), want)
        assert not (r.phase.astype(bool) & blocked).any()
        checked += 1
    assert checked >= 6


def test_phases_are_disjoint_and_reach_their_targets(oracle):
    rng = np.random.default_rng(55)
    for periodic in (0, 1):
        for _ in range(6):
            p1 = _random_case(rng, periodic)
            dims = {k: p1[k] for k in ("nx", "ny", "nz")}
            p2 = dict(_random_case(rng, periodic), **dims, target_solid_fraction=0.2)
            p3 = dict(_random_case(rng, periodic), **dims, target_solid_fraction=0.1)
            labels, rs = oracle.run_phases([p1, p2, p3])
            for k, r in enumerate(rs, start=1):
                assert int((labels == k).sum()) == r.solid_count
                if r.status == oracle.DONE:
                    assert r.solid_count == r.target_count
            assert np.array_equal(labels == 1, rs[0].phase.reshape(labels.shape).astype(bool))


def test_blocked_list_indexed_equals_full_field(oracle):
    rng = np.random.default_rng(56)
    for periodic in (0, 1):
        for _ in range(8):
            p = _random_case(rng, periodic)
            blocked = rng.random((p["nz"], p["ny"], p["nx"])) < 0.25
            a, b = oracle.run(p, blocked=blocked), oracle.run_fullfield(p, blocked=blocked)
            assert np.array_equal(a.phase, b.phase)
            assert (a.solid_count, a.steps, a.status, a.front_size) == \
                   (b.solid_count, b.steps, b.status, b.front_size)


# --------------------------------------------------------------------------
# Interacting phases (R13): the phase grows into cells of earlier phases
# with the interaction probability of the direction's class
# --------------------------------------------------------------------------
def _labels(rng, shape, n_labels, frac):
    """Random labels 1..n_labels on about `frac` of the cells, 0 elsewhere."""
    lab = rng.integers(1, n_labels + 1, size=shape).astype(np.uint8)
    lab[rng.random(shape) >= frac] = 0
    return lab


def test_interaction_zero_is_the_independent_phase(oracle):
    rng = np.random.default_rng(61)
    for periodic in (0, 1):
        for _ in range(8):
            p = _random_case(rng, periodic)
            lab = _labels(rng, (p["nz"], p["ny"], p["nx"]), 2, 0.3)
            a = oracle.run(p, blocked=lab)
            b = oracle.run(p, blocked=lab, inter=np.zeros((2, 3)))
            assert np.array_equal(a.phase, b.phase)
            assert (a.solid_count, a.steps, a.status, a.front_size) == \
                   (b.solid_count, b.steps, b.status, b.front_size)


def test_interaction_list_indexed_equals_full_field(oracle):
    rng = np.random.default_rng(62)
    for periodic in (0, 1):
        for _ in range(10):
            p = _random_case(rng, periodic)
            lab = _labels(rng, (p["nz"], p["ny"], p["nx"]), 3, 0.4)
            inter = rng.uniform(0.0, 0.6, size=(3, 3)) * (rng.random((3, 3)) < 0.7)
            a = oracle.run(p, blocked=lab, inter=inter)
            b = oracle.run_fullfield(p, blocked=lab, inter=inter)
            assert np.array_equal(a.phase, b.phase)
            assert (a.solid_count, a.steps, a.status, a.front_size) == \
                   (b.solid_count, b.steps, b.status, b.front_size)


def test_interaction_unit_probability_is_a_geodesic_dilation(oracle):
    # G = 0 and I = 1 towards label 1 only: the phase never grows into void
    # cells, and after k steps it is its seeds dilated k times (26-neighbour
    # steps) through the cells of label 1; label-2 cells stay blocked.
    rng = np.random.default_rng(63)
    checked = 0
    for trial in range(14):
        nx, ny, nz = (int(v) for v in rng.integers(5, 13, size=3))
        n = nx * ny * nz
        k = int(rng.integers(1, 4))
        lab = _labels(rng, (nz, ny, nx), 2, 0.7)
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.04, target_count=n, seed=trial, max_steps=k)
        cand = oracle.seed_candidates(p, blocked=lab)
        if cand.size == 0:
            continue
        want = np.zeros(n, bool)
        want[cand] = True
        want = want.reshape(nz, ny, nx)
        for _ in range(k):
            want |= ndimage.binary_dilation(want, structure=np.ones((3, 3, 3), bool)) & (lab == 1)
        r = oracle.run(p, blocked=lab, inter=np.array([[1.0, 1.0, 1.0], [0.0, 0.0, 0.0]]))
        assert np.array_equal(r.phase.astype(bool), want), trial
        assert not (r.phase.astype(bool) & (lab == 2)).any()
        checked += 1
    assert checked >= 6


def test_interaction_front_matches_bruteforce(oracle):
    # Active: a neighbour that is void, or of a label whose I is positive for
    # that direction's class.
    rng = np.random.default_rng(64)
    dirs, dcls = oracle.directions()
    for _ in range(20):
        nx, ny, nz = (int(v) for v in rng.integers(3, 11, size=3))
        lab = _labels(rng, (nz, ny, nx), 2, 0.4)
        inter = np.array([[0.5, 0.0, 0.0], [0.0, 0.0, 0.3]])   # label 1: faces, label 2: corners
        phase = (rng.random((nz, ny, nx)) < 0.5) & (lab == 0)
        ok = np.zeros((nz, ny, nx), bool)
        for (dx, dy, dz), c in zip(dirs, dcls):
            growable = (~phase & (lab == 0)) | (~phase & (lab >= 1) & (inter[np.maximum(lab, 1) - 1, c] > 0))
            pad = np.pad(growable, 1, constant_values=False)
            ok |= pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        got = oracle.front(dict(nx=nx, ny=ny, nz=nz, target_solid_fraction=0.5),
                           phase.astype(np.uint8), blocked=lab, inter=inter)
        assert np.array_equal(got, np.flatnonzero(phase & ok))


@pytest.mark.parametrize("cls", [0, 2])
def test_interaction_first_step_rate(oracle, cls):
    # Seeds on a slab of void cells facing a label-1 slab, G = 0: the step-0
    # entries into the label-1 slab are Bernoulli trials with p = floor(I 2^32) / 2^32
    # for the directions of one class (no Eq. 1 factor).
    prob = 0.15
    inter = np.zeros((1, 3))
    inter[0, cls] = prob
    dirs, dcls = oracle.directions()
    hits = trials = 0
    for seed in range(60):
        nx = ny = 16
        nz = 4
        lab = np.zeros((nz, ny, nx), np.uint8)
        lab[2:] = 1                                    # z >= 2: phase 1
        p = dict(nx=nx, ny=ny, nz=nz, cd=0.03, spacing_s=4, target_count=nx * ny * nz,
                 seed=seed, max_steps=1)
        seeds = np.zeros(nx * ny * nz, bool)
        seeds[oracle.seed_candidates(p, blocked=lab)] = True
        seeds = seeds.reshape(nz, ny, nx)
        r = oracle.run(p, blocked=lab, inter=inter)
        grown = r.phase.astype(bool) & (lab == 1)
        # attempts: (seed, direction of the class) pairs that land in the slab
        # with distinct targets -- spacing 4 keeps the targets of different
        # seeds apart for faces and corners
        s_idx = np.argwhere(seeds)
        placed = r.phase.astype(bool) & (lab == 0)
        s_idx = [t for t in s_idx if placed[tuple(t)]]
        for z, y, x in s_idx:
            for (dx, dy, dz), c in zip(dirs, dcls):
                zz, yy, xx = z + dz, y + dy, x + dx
                if c == cls and 0 <= xx < nx and 0 <= yy < ny and 0 <= zz < nz and lab[zz, yy, xx] == 1:
                    trials += 1
        hits += int(grown.sum())
    p_exact = np.floor(prob * 2**32) / 2**32
    z = (hits - trials * p_exact) / np.sqrt(trials * p_exact * (1 - p_exact))
    assert trials > 100 and abs(z) < 5, (hits, trials)


def test_interacting_phases_partition_and_reach_their_targets(oracle):
    rng = np.random.default_rng(65)
    for periodic in (0, 1):
        for _ in range(5):
            p1 = _random_case(rng, periodic)
            dims = {k: p1[k] for k in ("nx", "ny", "nz")}
            p2 = dict(_random_case(rng, periodic), **dims, target_solid_fraction=0.3)
            p3 = dict(_random_case(rng, periodic), **dims, target_solid_fraction=0.15)
            spec = [None, {1: (0.4, 0.2, 0.1)}, {1: (0.2, 0.0, 0.0), 2: (0.0, 0.3, 0.3)}]
            labels, rs = oracle.run_phases([p1, p2, p3], spec)
            indep, _ = oracle.run_phases([p1, p2, p3])
            # the last phase's cells are exactly its own realization
            assert np.array_equal(labels == 3, rs[2].phase.reshape(labels.shape).astype(bool))
            for k, r in enumerate(rs, start=1):
                if r.status == oracle.DONE:
                    assert r.solid_count == r.target_count
            # entering earlier phases only takes cells from them
            assert int((labels == 1).sum()) <= rs[0].solid_count
            assert np.array_equal(indep == 1, rs[0].phase.reshape(labels.shape).astype(bool))
            assert not ((labels == 1) & (indep != 1)).any()
