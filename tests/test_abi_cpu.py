"""The C-ABI library builds, loads and exports every declared entry point;
its host-side parameter logic agrees with the oracle.  No GPU needed: only
functions that touch no device are called."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2602_11734_gb300 import build as B
from paper_2602_11734_gb300 import qsgs as Q
from paper_2602_11734_gb300 import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return Q.load_library()


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(qsgs_\w+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "qsgs_create" in syms and "qsgs_grow_until" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_version_and_strerror(lib):
    assert lib.qsgs_version() >= 100
    for code in (0, 1, 2, 3, -1, -2, -3, -4, -5, -6, 12345):
        assert isinstance(Q.strerror(code), str) and Q.strerror(code)


def test_check_params_matches_oracle(lib, oracle):
    rng = np.random.default_rng(8)
    cases = [workloads.small_64(), workloads.single_400()] + workloads.sweep_500()[:3]
    cases += [workloads.random_small(rng) for _ in range(200)]
    for p in cases:
        assert Q.qsgs_check_params(p) == oracle.targets(p)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(cd=1.5), dict(cd=-0.1), dict(g_face=2.0),
                                 dict(g_corner=float("nan")), dict(target_count=10**6),
                                 dict(target_solid_fraction=1.2),
                                 dict(nx=2**11, ny=2**11, nz=2**10)])
def test_invalid_params_rejected(lib, bad):
    p = dict(nx=8, ny=8, nz=8, target_solid_fraction=0.5)
    p.update(bad)
    with pytest.raises(Q.QsgsError) as e:
        Q.qsgs_check_params(p)
    assert e.value.code == Q.QSGS_ERR_INVALID
    assert Q.qsgs_workspace_bytes(p) == 0


def test_workspace_bytes(lib):
    def words(p):
        return ((p["nx"] + 31) // 32) * p["ny"] * p["nz"]

    for p in (workloads.small_64(), workloads.single_400(), workloads.fig3_size(1000, True),
              workloads.fig3_size(1000, False)):
        b = Q.qsgs_workspace_bytes(p)
        # grid + two claim grids + the candidate word list, 4 B per word each
        assert b >= 16 * words(p), p
        # nothing per voxel: the seed arrays scale with the candidate count
        n = p["nx"] * p["ny"] * p["nz"]
        cand = n * p["cd"] + 8 * (n * p["cd"]) ** 0.5 + 4096
        assert b <= 17 * words(p) + 40 * cand + 8 * (n // max(2, p["spacing_s"]) ** 3) + (1 << 20), p
    small = Q.qsgs_workspace_bytes(workloads.small_64())
    with_spacing = Q.qsgs_workspace_bytes(dict(workloads.small_64(), spacing_s=5))
    assert with_spacing > small
    # every voxel a candidate (cd = 1): the capacity is N itself
    dense = dict(workloads.small_64(), cd=1.0, spacing_s=3)
    assert Q.qsgs_workspace_bytes(dense) >= 64**3 * (4 + 4 + 1 + 4)


def test_create_rejects_bad_workspace_without_touching_the_device(lib):
    p = Q.make_params(workloads.small_64())
    need = lib.qsgs_workspace_bytes(ctypes.byref(p))
    h = ctypes.c_void_p()
    rc = lib.qsgs_create(ctypes.byref(p), None, need, None, ctypes.byref(h))
    assert rc == Q.QSGS_ERR_WORKSPACE and not h.value
    rc = lib.qsgs_create(ctypes.byref(p), ctypes.c_void_p(256 * 7), need - 1, None, ctypes.byref(h))
    assert rc == Q.QSGS_ERR_WORKSPACE
    rc = lib.qsgs_create(ctypes.byref(p), ctypes.c_void_p(256 * 7 + 8), need, None, ctypes.byref(h))
    assert rc == Q.QSGS_ERR_WORKSPACE
    bad = Q.make_params(dict(workloads.small_64(), cd=3.0))
    rc = lib.qsgs_create(ctypes.byref(bad), ctypes.c_void_p(256), 1 << 30, None, ctypes.byref(h))
    assert rc == Q.QSGS_ERR_INVALID
    assert lib.qsgs_create(ctypes.byref(p), None, 0, None, None) == Q.QSGS_ERR_INVALID


def test_null_handles_are_rejected(lib):
    s = Q.QsgsStats()
    assert lib.qsgs_seed(None) == Q.QSGS_ERR_INVALID
    assert lib.qsgs_grow_until(None, 0, ctypes.byref(s)) == Q.QSGS_ERR_INVALID
    assert lib.qsgs_query(None, ctypes.byref(s)) == Q.QSGS_ERR_INVALID
    assert lib.qsgs_fetch(None, None, 0, 0, 0) == Q.QSGS_ERR_INVALID
    lib.qsgs_destroy(None)


def test_periodic_params_checked_like_the_oracle(lib, oracle):
    for dims, ok in (((3, 3, 3), True), ((2, 9, 9), False), ((9, 1, 9), False), ((40, 33, 3), True)):
        p = dict(nx=dims[0], ny=dims[1], nz=dims[2], cd=0.01, target_solid_fraction=0.5, periodic=1)
        if ok:
            Q.qsgs_check_params(p)
            assert Q.qsgs_workspace_bytes(p) > 0
        else:
            with pytest.raises(Q.QsgsError) as e:
                Q.qsgs_check_params(p)
            assert e.value.code == Q.QSGS_ERR_INVALID
            with pytest.raises(Exception):
                oracle.run(p)
    with pytest.raises(Q.QsgsError):
        Q.qsgs_check_params(dict(nx=8, ny=8, nz=8, target_solid_fraction=0.5, periodic=2))


def test_every_handle_call_rejects_a_null_handle(lib):
    """Each entry point that takes a handle returns QSGS_ERR_INVALID for
    NULL before it touches a device (include/qsgs.h: no exceptions, no
    crash across the ABI)."""
    inv = Q.QSGS_ERR_INVALID
    s = Q.QsgsStats()
    prof = (Q.QsgsProfileEntry * 8)()
    ms = ctypes.c_double()
    probs = (ctypes.c_double * 3)(0.1, 0.1, 0.1)
    assert lib.qsgs_set_profiling(None, 1) == inv
    assert lib.qsgs_profile(None, prof, 8) == inv
    assert lib.qsgs_set_grow_blocks(None, 0) == inv
    assert lib.qsgs_set_grow_tile(None, 1) == inv
    assert lib.qsgs_set_mode(None, 0) == inv
    assert lib.qsgs_set_spin_limit(None, 0) == inv
    assert lib.qsgs_set_blocked(None, None) == inv
    assert lib.qsgs_set_interaction(None, None, probs, 1, None, 0) == inv
    assert lib.qsgs_fetch_label(None, None, 0, 1) == inv
    assert lib.qsgs_fetch_or(None, None, 0) == inv
    assert lib.qsgs_time_grow(None, 0, 1, ctypes.byref(ms)) == inv
    assert lib.qsgs_batch_set_members(None, None, 0) == inv
    assert lib.qsgs_batch_seed(None) == inv
    assert lib.qsgs_batch_advance(None, 0) == inv
    assert lib.qsgs_batch_query(None, ctypes.byref(s), 1) == inv
    assert lib.qsgs_batch_run(None, 0, ctypes.byref(s), 1) == inv
    assert lib.qsgs_batch_set_grow_blocks(None, 0) == inv
    assert lib.qsgs_batch_set_grow_tile(None, 1) == inv
    assert lib.qsgs_batch_set_profiling(None, 1) == inv
    assert lib.qsgs_batch_profile(None, prof, 8) == inv
    lib.qsgs_batch_destroy(None)


def test_batch_and_interaction_sizing_on_the_host(lib):
    # batch workspace: members 1 .. 1024, words below 2^32; 0 = invalid
    assert lib.qsgs_batch_workspace_bytes(0, 1000) == 0
    assert lib.qsgs_batch_workspace_bytes(1025, 1000) == 0
    assert lib.qsgs_batch_workspace_bytes(4, 1 << 32) == 0
    a = lib.qsgs_batch_workspace_bytes(4, 1000)
    b = lib.qsgs_batch_workspace_bytes(4, 2000)
    assert a > 0 and b - a >= 4000  # one u32 list entry per word
    h = ctypes.c_void_p()
    assert lib.qsgs_batch_create(0, 10, None, 0, None, ctypes.byref(h)) == Q.QSGS_ERR_INVALID
    assert lib.qsgs_batch_create(4, 1000, None, a, None, ctypes.byref(h)) == Q.QSGS_ERR_WORKSPACE
    assert lib.qsgs_batch_create(4, 1000, ctypes.c_void_p(256), a - 1, None,
                                 ctypes.byref(h)) == Q.QSGS_ERR_WORKSPACE
    assert lib.qsgs_batch_create(4, 1000, None, a, None, None) == Q.QSGS_ERR_INVALID
    # interaction scratch: four packed grids (blocked + three per-class
    # enterable grids) and 256 x 3 thresholds
    for p in (workloads.small_64(), dict(workloads.small_64(), nx=70, ny=33, nz=29)):
        words = ((p["nx"] + 31) // 32) * p["ny"] * p["nz"]
        assert lib.qsgs_interaction_bytes(ctypes.byref(Q.make_params(p))) == 16 * words + 3072
    bad = Q.make_params(dict(workloads.small_64(), cd=2.0))
    assert lib.qsgs_interaction_bytes(ctypes.byref(bad)) == 0


def test_snapshot_size_is_header_state_and_grid(lib):
    # 256-byte header + 256-byte run state + the packed grid; host only.
    for p in (workloads.small_64(), workloads.single_400(),
              dict(workloads.small_64(), nx=33, ny=5, nz=7)):
        words = (p["nx"] + 31) // 32 * p["ny"] * p["nz"]
        assert Q.qsgs_snapshot_bytes(p) == 512 + 4 * words
    assert Q.qsgs_snapshot_bytes(dict(workloads.small_64(), nx=0)) == 0
