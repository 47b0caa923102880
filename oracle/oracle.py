"""ctypes wrapper of the CPU oracle (qsgs_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by the smoke check in
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``; the product
package never imports it.  It shares no code with the CUDA path: it builds
and loads its own plain-C shared library.

Parameters are plain dicts with the keys of ``oq_params`` (nx, ny, nz, cd,
g_face, g_edge, g_corner, spacing_s, target_solid_fraction, target_count,
seed, max_steps); missing keys take the defaults below.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsgs_oracle.c")
_HDR = os.path.join(_HERE, "qsgs_oracle.h")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libqsgs_oracle.so")

DONE, STALLED, MAX_STEPS = 0, 1, 2

DEFAULTS = dict(nx=8, ny=8, nz=8, cd=0.0, g_face=0.0, g_edge=0.0, g_corner=0.0,
                spacing_s=0, target_solid_fraction=0.0, target_count=0, seed=0,
                max_steps=0, periodic=0)


class OqParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_uint32), ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32),
                ("cd", ctypes.c_double), ("g_face", ctypes.c_double),
                ("g_edge", ctypes.c_double), ("g_corner", ctypes.c_double),
                ("spacing_s", ctypes.c_uint32), ("target_solid_fraction", ctypes.c_double),
                ("target_count", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("max_steps", ctypes.c_uint32), ("periodic", ctypes.c_uint32),
                ("blocked", ctypes.c_void_p), ("inter", ctypes.c_void_p),
                ("n_labels", ctypes.c_uint32)]


class OqStepLog(ctypes.Structure):
    _fields_ = [("t", ctypes.c_uint32), ("solid_before", ctypes.c_uint64),
                ("front", ctypes.c_uint64), ("claimed", ctypes.c_uint64),
                ("thr", ctypes.c_uint64 * 3)]


class OqSummary(ctypes.Structure):
    _fields_ = [("solid_count", ctypes.c_uint64), ("target_count", ctypes.c_uint64),
                ("front_size", ctypes.c_uint64), ("n_candidates", ctypes.c_uint64),
                ("n_accepted", ctypes.c_uint64), ("steps", ctypes.c_uint32),
                ("status", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no target-specific flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH) or
             max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)) > os.path.getmtime(_LIB_PATH))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            i32p = ctypes.POINTER(ctypes.c_int32)
            P = ctypes.POINTER(OqParams)
            L.oq_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.oq_philox4x32_10.restype = None
            L.oq_directions.argtypes = [i32p, i32p]
            L.oq_directions.restype = None
            L.oq_targets.argtypes = [P, u64p, u64p, u64p]
            L.oq_targets.restype = ctypes.c_int
            L.oq_threshold.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            L.oq_threshold.restype = ctypes.c_uint64
            L.oq_seed_candidates.argtypes = [P, u32p, ctypes.c_uint64]
            L.oq_seed_candidates.restype = ctypes.c_uint64
            L.oq_spacing.argtypes = [P, u32p, ctypes.c_uint64, u8p]
            L.oq_spacing.restype = ctypes.c_int
            L.oq_front.argtypes = [P, u8p, u32p]
            L.oq_front.restype = ctypes.c_uint64
            L.oq_run.argtypes = [P, u8p, ctypes.POINTER(OqStepLog), ctypes.c_uint32,
                                 ctypes.POINTER(OqSummary)]
            L.oq_run.restype = ctypes.c_int
            L.oq_run_fullfield.argtypes = [P, u8p, ctypes.POINTER(OqSummary)]
            L.oq_run_fullfield.restype = ctypes.c_int
            _lib = L
    return _lib


def _params(p: dict, blocked=None, inter=None) -> OqParams:
    """Parameters; ``blocked`` (optional, N bytes, x fastest): labels of
    earlier phases, 0 = unassigned (R12); ``inter`` (optional, (n_labels, 3)):
    interaction probabilities I^{n,m} per label m = 1.. and class (R13).
    The returned struct keeps the arrays alive."""
    q = dict(DEFAULTS)
    unknown = set(p) - set(DEFAULTS)
    if unknown:
        raise KeyError(f"unknown parameter(s) {sorted(unknown)}")
    q.update(p)
    P = OqParams(**q)
    if blocked is not None:
        arr = np.ascontiguousarray(blocked, dtype=np.uint8).reshape(-1)
        if arr.size != P.nx * P.ny * P.nz:
            raise ValueError("blocked must hold one byte per voxel")
        P.blocked = arr.ctypes.data
        P._keep = arr
    if inter is not None:
        tab = np.ascontiguousarray(inter, dtype=np.float64).reshape(-1, 3)
        P.inter = tab.ctypes.data
        P.n_labels = tab.shape[0]
        P._keep_inter = tab
    return P


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: ctr = 4 u32 words, key = 2 u32 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oq_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                           _ptr(out, ctypes.c_uint32))
    return out


def directions():
    """(dirs int32 (26,3) as (dx,dy,dz), class int32 (26,))."""
    d = np.zeros(78, dtype=np.int32)
    c = np.zeros(26, dtype=np.int32)
    lib().oq_directions(_ptr(d, ctypes.c_int32), _ptr(c, ctypes.c_int32))
    return d.reshape(26, 3), c


def targets(p: dict):
    """(Nt, T_seed, (T_face, T_edge, T_corner)); raises ValueError if invalid."""
    nt, ts = ctypes.c_uint64(), ctypes.c_uint64()
    tr = (ctypes.c_uint64 * 3)()
    rc = lib().oq_targets(ctypes.byref(_params(p)), ctypes.byref(nt), ctypes.byref(ts), tr)
    if rc != 0:
        raise ValueError(f"invalid parameters (rc={rc})")
    return nt.value, ts.value, tuple(tr)


def threshold(t_ref: int, nt: int, c: int) -> int:
    return int(lib().oq_threshold(t_ref, nt, c))


def seed_candidates(p: dict, blocked=None, inter=None) -> np.ndarray:
    P = _params(p, blocked, inter)
    n = lib().oq_seed_candidates(ctypes.byref(P), None, 0)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    lib().oq_seed_candidates(ctypes.byref(P), _ptr(out, ctypes.c_uint32), n)
    return out[:n]


def spacing(p: dict, cand: np.ndarray) -> np.ndarray:
    c = np.ascontiguousarray(cand, dtype=np.uint32)
    acc = np.zeros(max(len(c), 1), dtype=np.uint8)
    rc = lib().oq_spacing(ctypes.byref(_params(p)), _ptr(c, ctypes.c_uint32), len(c),
                          _ptr(acc, ctypes.c_uint8))
    if rc != 0:
        raise MemoryError("oracle spacing failed")
    return acc[:len(c)].astype(bool)


def front(p: dict, phase: np.ndarray, blocked=None, inter=None) -> np.ndarray:
    ph = np.ascontiguousarray(phase, dtype=np.uint8).reshape(-1)
    out = np.zeros(max(ph.size, 1), dtype=np.uint32)
    P = _params(p, blocked, inter)
    n = lib().oq_front(ctypes.byref(P), _ptr(ph, ctypes.c_uint8), _ptr(out, ctypes.c_uint32))
    return out[:n]


@dataclass
class Result:
    phase: np.ndarray          # uint8 (nz, ny, nx), 1 = solid
    solid_count: int
    target_count: int
    front_size: int
    n_candidates: int
    n_accepted: int
    steps: int
    status: int
    log: np.ndarray | None     # structured: t, solid_before, front, claimed, thr (3,)


_LOG_DTYPE = np.dtype([("t", np.uint32), ("solid_before", np.uint64), ("front", np.uint64),
                       ("claimed", np.uint64), ("thr", np.uint64, (3,))], align=True)
assert _LOG_DTYPE.itemsize == ctypes.sizeof(OqStepLog)


def _result(P: OqParams, phase: np.ndarray, s: OqSummary, log) -> Result:
    return Result(phase=phase.reshape(P.nz, P.ny, P.nx), solid_count=s.solid_count,
                  target_count=s.target_count, front_size=s.front_size,
                  n_candidates=s.n_candidates, n_accepted=s.n_accepted, steps=s.steps,
                  status=s.status, log=log)


def run(p: dict, log_cap: int = 100000, blocked=None, inter=None) -> Result:
    """One realization by Algorithm 3 (list-indexed growth); ``blocked``:
    labels of earlier phases (R12); ``inter``: their interaction
    probabilities (R13)."""
    P = _params(p, blocked, inter)
    n = P.nx * P.ny * P.nz
    phase = np.zeros(n, dtype=np.uint8)
    log = np.zeros(log_cap, dtype=_LOG_DTYPE)
    s = OqSummary()
    rc = lib().oq_run(ctypes.byref(P), _ptr(phase, ctypes.c_uint8),
                      log.ctypes.data_as(ctypes.POINTER(OqStepLog)), log_cap, ctypes.byref(s))
    if rc != 0:
        raise ValueError(f"oracle run failed (rc={rc})")
    return _result(P, phase, s, log[:min(s.steps, log_cap)])


def run_fullfield(p: dict, blocked=None, inter=None) -> Result:
    """The same realization by the full-field sweep of Algorithm 2."""
    P = _params(p, blocked, inter)
    n = P.nx * P.ny * P.nz
    phase = np.zeros(n, dtype=np.uint8)
    s = OqSummary()
    rc = lib().oq_run_fullfield(ctypes.byref(P), _ptr(phase, ctypes.c_uint8), ctypes.byref(s))
    if rc != 0:
        raise ValueError(f"oracle run failed (rc={rc})")
    return _result(P, phase, s, None)


def run_phases(phases: list, interactions=None) -> tuple:
    """Sec. 2.1 steps 4-5: phase k (k = 1, 2, ...) is generated on the cells
    no earlier phase holds (R12) -- or, when interactions[k - 1] is a dict
    {m: (I_face, I_edge, I_corner)}, also enters cells of the earlier phases
    m listed there (R13), which become phase k's.  The label map has k on
    phase k's cells and 0 on the matrix.  Returns (labels (nz, ny, nx)
    uint8, [Result of every phase])."""
    p0 = dict(DEFAULTS, **phases[0])
    shape = (p0["nz"], p0["ny"], p0["nx"])
    labels = np.zeros(shape, dtype=np.uint8)
    results = []
    for k, p in enumerate(phases, start=1):
        spec = interactions[k - 1] if interactions else None
        inter = None
        if spec:
            inter = np.zeros((k - 1, 3))
            for m, probs in spec.items():
                if not 1 <= m < k:
                    raise ValueError(f"phase {k} can only enter earlier phases, not {m}")
                inter[m - 1] = probs
        r = run(p, blocked=labels, inter=inter)
        labels[r.phase.astype(bool)] = k
        results.append(r)
    return labels, results
