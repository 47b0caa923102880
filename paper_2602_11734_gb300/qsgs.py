"""Python binding of libqsgs (include/qsgs.h).

Argument marshalling only: every step of generation runs in the CUDA
kernels behind the C ABI.  PyTorch supplies device memory (the workspace
and output tensors) and CUDA streams.  There is no CPU fallback: if the
library is missing or no CUDA device is present, calls raise.

The functions ``qsgs_*`` mirror the C entry points one to one; the
``Generator`` class is a convenience wrapper that owns a workspace tensor
and a stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
# QSGS_LIBRARY overrides the library path (e.g. a build with other tuning).
LIB_PATH = os.environ.get("QSGS_LIBRARY") or os.path.join(PKG, "_build", "libqsgs.so")

QSGS_OK, QSGS_STALLED, QSGS_MAX_STEPS, QSGS_RUNNING = 0, 1, 2, 3
QSGS_ERR_INVALID, QSGS_ERR_WORKSPACE, QSGS_ERR_CUDA = -1, -2, -3
QSGS_ERR_TIMEOUT, QSGS_ERR_STATE, QSGS_ERR_NOMEM = -4, -5, -6
QSGS_FMT_U8, QSGS_FMT_PACKED = 0, 1
QSGS_DST_HOST, QSGS_DST_DEVICE, QSGS_DST_HOST_MAPPED = 0, 1, 2
QSGS_MODE_LIETS, QSGS_MODE_FULLFIELD = 0, 1

PARAM_KEYS = ("nx", "ny", "nz", "cd", "g_face", "g_edge", "g_corner", "spacing_s",
              "target_solid_fraction", "target_count", "seed", "max_steps", "periodic")


class QsgsParams(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_uint32), ("ny", ctypes.c_uint32), ("nz", ctypes.c_uint32),
                ("cd", ctypes.c_double), ("g_face", ctypes.c_double),
                ("g_edge", ctypes.c_double), ("g_corner", ctypes.c_double),
                ("spacing_s", ctypes.c_uint32), ("target_solid_fraction", ctypes.c_double),
                ("target_count", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("max_steps", ctypes.c_uint32), ("periodic", ctypes.c_uint32)]


class QsgsStats(ctypes.Structure):
    _fields_ = [("solid_count", ctypes.c_uint64), ("target_count", ctypes.c_uint64),
                ("front_size", ctypes.c_uint64), ("n_candidates", ctypes.c_uint64),
                ("n_seeds", ctypes.c_uint64), ("sum_front", ctypes.c_uint64),
                ("steps", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("launches", ctypes.c_uint64), ("sum_draws", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class QsgsProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class QsgsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqsgs.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"libqsgs not built ({path} missing); run "
                    "`python -m paper_2602_11734_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(path)
            vp, u64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)
            P, S = ctypes.POINTER(QsgsParams), ctypes.POINTER(QsgsStats)
            H = ctypes.c_void_p
            sig = {
                "qsgs_version": ([], ctypes.c_int),
                "qsgs_strerror": ([ctypes.c_int], ctypes.c_char_p),
                "qsgs_check_params": ([P, u64p, u64p, u64p], ctypes.c_int),
                "qsgs_workspace_bytes": ([P], ctypes.c_size_t),
                "qsgs_create": ([P, vp, ctypes.c_size_t, vp, ctypes.POINTER(H)], ctypes.c_int),
                "qsgs_seed": ([H], ctypes.c_int),
                "qsgs_grow_until": ([H, ctypes.c_uint32, S], ctypes.c_int),
                "qsgs_fetch": ([H, vp, ctypes.c_size_t, ctypes.c_int, ctypes.c_int], ctypes.c_int),
                "qsgs_query": ([H, S], ctypes.c_int),
                "qsgs_snapshot_bytes": ([P], ctypes.c_size_t),
                "qsgs_snapshot": ([H, vp, ctypes.c_size_t, ctypes.c_int], ctypes.c_int),
                "qsgs_restore": ([H, vp, ctypes.c_size_t, ctypes.c_int], ctypes.c_int),
                "qsgs_set_profiling": ([H, ctypes.c_int], ctypes.c_int),
                "qsgs_profile": ([H, ctypes.POINTER(QsgsProfileEntry), ctypes.c_int],
                                 ctypes.c_int),
                "qsgs_bench_philox": ([ctypes.c_uint64, vp, vp, ctypes.POINTER(ctypes.c_double)],
                                      ctypes.c_int),
                "qsgs_bench_l2_read": ([vp, ctypes.c_size_t, ctypes.c_uint32, vp, vp,
                                        ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
                "qsgs_bench_l2_atomic": ([vp, ctypes.c_size_t, ctypes.c_uint64, vp,
                                          ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
                "qsgs_destroy": ([H], None),
                "qsgs_set_grow_blocks": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_set_grow_tile": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_set_mode": ([H, ctypes.c_int], ctypes.c_int),
                "qsgs_set_blocked": ([H, ctypes.c_void_p], ctypes.c_int),
                "qsgs_interaction_bytes": ([P], ctypes.c_size_t),
                "qsgs_set_interaction": ([H, vp, ctypes.POINTER(ctypes.c_double), ctypes.c_uint32,
                                          vp, ctypes.c_size_t], ctypes.c_int),
                "qsgs_set_spin_limit": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_fetch_label": ([H, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint8],
                                     ctypes.c_int),
                "qsgs_fetch_or": ([H, ctypes.c_void_p, ctypes.c_size_t], ctypes.c_int),
                "qsgs_time_grow": ([H, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
                "qsgs_front_count_static": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
                "qsgs_batch_workspace_bytes": ([ctypes.c_uint32, ctypes.c_uint64], ctypes.c_size_t),
                "qsgs_batch_create": ([ctypes.c_uint32, ctypes.c_uint64, vp, ctypes.c_size_t, vp,
                                       ctypes.POINTER(H)], ctypes.c_int),
                "qsgs_batch_set_members": ([H, ctypes.POINTER(H), ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_seed": ([H], ctypes.c_int),
                "qsgs_batch_advance": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_query": ([H, S, ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_run": ([H, ctypes.c_uint32, S, ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_set_grow_blocks": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_set_grow_tile": ([H, ctypes.c_uint32], ctypes.c_int),
                "qsgs_batch_set_profiling": ([H, ctypes.c_int], ctypes.c_int),
                "qsgs_batch_profile": ([H, ctypes.POINTER(QsgsProfileEntry), ctypes.c_int],
                                       ctypes.c_int),
                "qsgs_batch_destroy": ([H], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return load_library().qsgs_strerror(code).decode()
    except RuntimeError:
        return f"code {code}"


def make_params(p: dict) -> QsgsParams:
    unknown = set(p) - set(PARAM_KEYS)
    if unknown:
        raise KeyError(f"unknown parameter(s) {sorted(unknown)}")
    q = dict(nx=1, ny=1, nz=1, cd=0.0, g_face=0.0, g_edge=0.0, g_corner=0.0, spacing_s=0,
             target_solid_fraction=0.0, target_count=0, seed=0, max_steps=0, periodic=0)
    q.update(p)
    return QsgsParams(**q)


# ---- thin one-to-one wrappers of the C entry points -----------------------
def qsgs_check_params(p: dict):
    """(Nt, T_seed, (T_face, T_edge, T_corner)); raises QsgsError if invalid."""
    nt, ts = ctypes.c_uint64(), ctypes.c_uint64()
    tr = (ctypes.c_uint64 * 3)()
    rc = load_library().qsgs_check_params(ctypes.byref(make_params(p)), ctypes.byref(nt),
                                          ctypes.byref(ts), tr)
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_check_params")
    return nt.value, ts.value, tuple(tr)


def qsgs_workspace_bytes(p: dict) -> int:
    return int(load_library().qsgs_workspace_bytes(ctypes.byref(make_params(p))))


def qsgs_create(p: dict, workspace_ptr: int, nbytes: int, stream_ptr: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    rc = load_library().qsgs_create(ctypes.byref(make_params(p)), ctypes.c_void_p(workspace_ptr),
                                    nbytes, ctypes.c_void_p(stream_ptr), ctypes.byref(h))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_create")
    return h


def qsgs_seed(h) -> None:
    rc = load_library().qsgs_seed(h)
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_seed")


def qsgs_grow_until(h, max_steps: int = 0) -> tuple[int, dict]:
    s = QsgsStats()
    rc = load_library().qsgs_grow_until(h, max_steps, ctypes.byref(s))
    if rc < 0:
        raise QsgsError(rc, "qsgs_grow_until")
    return rc, s.as_dict()


def qsgs_fetch(h, dst_ptr: int, nbytes: int, fmt: int, dst_is_device: int) -> None:
    """dst_is_device: QSGS_DST_HOST (or False), QSGS_DST_DEVICE (or True) or
    QSGS_DST_HOST_MAPPED."""
    rc = load_library().qsgs_fetch(h, ctypes.c_void_p(dst_ptr), nbytes, fmt, int(dst_is_device))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_fetch")


def qsgs_query(h) -> dict:
    s = QsgsStats()
    rc = load_library().qsgs_query(h, ctypes.byref(s))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_query")
    return s.as_dict()


def qsgs_snapshot_bytes(p: dict) -> int:
    return int(load_library().qsgs_snapshot_bytes(ctypes.byref(make_params(p))))


def qsgs_snapshot(h, dst_ptr: int, nbytes: int, dst_kind: int) -> None:
    rc = load_library().qsgs_snapshot(h, ctypes.c_void_p(dst_ptr), nbytes, dst_kind)
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_snapshot")


def qsgs_restore(h, src_ptr: int, nbytes: int, src_kind: int) -> None:
    rc = load_library().qsgs_restore(h, ctypes.c_void_p(src_ptr), nbytes, src_kind)
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_restore")


def qsgs_set_profiling(h, enable: bool) -> None:
    rc = load_library().qsgs_set_profiling(h, int(enable))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_set_profiling")


def qsgs_profile(h) -> dict:
    """{kernel class: (launches, total_ms)} of the event profiler."""
    buf = (QsgsProfileEntry * 16)()
    n = load_library().qsgs_profile(h, buf, 16)
    if n < 0:
        raise QsgsError(n, "qsgs_profile")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(min(n, 16))}


def qsgs_bench_philox(n_blocks: int, dev_out_ptr: int, stream_ptr: int) -> float:
    """Milliseconds the GPU needs for n_blocks Philox4x32-10 blocks."""
    ms = ctypes.c_double()
    rc = load_library().qsgs_bench_philox(n_blocks, ctypes.c_void_p(dev_out_ptr),
                                          ctypes.c_void_p(stream_ptr), ctypes.byref(ms))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_bench_philox")
    return ms.value


def qsgs_bench_l2_read(buf_ptr: int, nbytes: int, passes: int, dev_out_ptr: int,
                       stream_ptr: int) -> float:
    """Milliseconds for ``passes`` reads of an L2-resident device buffer."""
    ms = ctypes.c_double()
    rc = load_library().qsgs_bench_l2_read(ctypes.c_void_p(buf_ptr), nbytes, passes,
                                           ctypes.c_void_p(dev_out_ptr),
                                           ctypes.c_void_p(stream_ptr), ctypes.byref(ms))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_bench_l2_read")
    return ms.value


def qsgs_bench_l2_atomic(buf_ptr: int, nbytes: int, n_ops: int, stream_ptr: int) -> float:
    """Milliseconds for n_ops scattered atomicOr reductions into a device buffer."""
    ms = ctypes.c_double()
    rc = load_library().qsgs_bench_l2_atomic(ctypes.c_void_p(buf_ptr), nbytes, n_ops,
                                             ctypes.c_void_p(stream_ptr), ctypes.byref(ms))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_bench_l2_atomic")
    return ms.value


def qsgs_destroy(h) -> None:
    if h:
        load_library().qsgs_destroy(h)


def qsgs_set_grow_blocks(h, blocks: int) -> None:
    rc = load_library().qsgs_set_grow_blocks(h, blocks)
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_set_grow_blocks")


def qsgs_time_grow(h, grow_blocks: int = 0, reps: int = 5) -> float:
    ms = ctypes.c_double()
    rc = load_library().qsgs_time_grow(h, grow_blocks, reps, ctypes.byref(ms))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_time_grow")
    return ms.value


def qsgs_front_count_static(grid_ptr: int, nx: int, ny: int, nz: int, stream_ptr: int = 0) -> int:
    """Front size of a packed device grid; allocates nothing (static scratch)."""
    out = ctypes.c_uint64()
    rc = load_library().qsgs_front_count_static(ctypes.c_void_p(grid_ptr), nx, ny, nz,
                                                ctypes.c_void_p(stream_ptr), ctypes.byref(out))
    if rc != QSGS_OK:
        raise QsgsError(rc, "qsgs_front_count_static")
    return out.value


def qsgs_version() -> int:
    return load_library().qsgs_version()


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise QsgsError(rc, where)
    return rc


def qsgs_batch_workspace_bytes(max_members: int, max_words: int) -> int:
    return int(load_library().qsgs_batch_workspace_bytes(max_members, max_words))


def qsgs_batch_create(max_members: int, max_words: int, workspace_ptr: int, nbytes: int,
                      stream_ptr: int):
    b = ctypes.c_void_p()
    _check(load_library().qsgs_batch_create(max_members, max_words, ctypes.c_void_p(workspace_ptr),
                                            nbytes, ctypes.c_void_p(stream_ptr), ctypes.byref(b)),
           "qsgs_batch_create")
    return b


def qsgs_batch_set_members(b, handles) -> None:
    arr = (ctypes.c_void_p * max(1, len(handles)))(*[h.value for h in handles])
    _check(load_library().qsgs_batch_set_members(b, arr, len(handles)), "qsgs_batch_set_members")


def qsgs_batch_seed(b) -> None:
    _check(load_library().qsgs_batch_seed(b), "qsgs_batch_seed")


def qsgs_batch_advance(b, max_steps: int = 0) -> None:
    _check(load_library().qsgs_batch_advance(b, max_steps), "qsgs_batch_advance")


def qsgs_batch_query(b, n: int) -> list[dict]:
    arr = (QsgsStats * max(1, n))()
    _check(load_library().qsgs_batch_query(b, arr, n), "qsgs_batch_query")
    return [arr[i].as_dict() for i in range(n)]


def qsgs_batch_set_grow_blocks(b, blocks: int) -> None:
    _check(load_library().qsgs_batch_set_grow_blocks(b, blocks), "qsgs_batch_set_grow_blocks")


def qsgs_set_grow_tile(h, chunks: int) -> None:
    _check(load_library().qsgs_set_grow_tile(h, chunks), "qsgs_set_grow_tile")


def qsgs_set_mode(h, mode: int) -> None:
    _check(load_library().qsgs_set_mode(h, mode), "qsgs_set_mode")


def qsgs_set_spin_limit(h, polls: int) -> None:
    _check(load_library().qsgs_set_spin_limit(h, polls), "qsgs_set_spin_limit")


def qsgs_set_blocked(h, dev_ptr: int) -> None:
    _check(load_library().qsgs_set_blocked(h, ctypes.c_void_p(dev_ptr or None)),
           "qsgs_set_blocked")


def qsgs_interaction_bytes(p: dict) -> int:
    return int(load_library().qsgs_interaction_bytes(ctypes.byref(make_params(p))))


def qsgs_set_interaction(h, labels_ptr: int, probs, scratch_ptr: int, scratch_bytes: int) -> None:
    """probs: rows (I_face, I_edge, I_corner) of the labels 1, 2, ...; labels_ptr
    0 clears the interaction."""
    rows = [tuple(float(v) for v in r) for r in (probs if probs is not None else [])]
    arr = (ctypes.c_double * max(1, 3 * len(rows)))(*[v for r in rows for v in r])
    _check(load_library().qsgs_set_interaction(h, ctypes.c_void_p(labels_ptr or None), arr,
                                               len(rows), ctypes.c_void_p(scratch_ptr or None),
                                               scratch_bytes), "qsgs_set_interaction")


def qsgs_fetch_label(h, dev_ptr: int, nbytes: int, label: int) -> None:
    _check(load_library().qsgs_fetch_label(h, ctypes.c_void_p(dev_ptr), nbytes, label),
           "qsgs_fetch_label")


def qsgs_fetch_or(h, dev_ptr: int, nbytes: int) -> None:
    _check(load_library().qsgs_fetch_or(h, ctypes.c_void_p(dev_ptr), nbytes), "qsgs_fetch_or")


def qsgs_batch_set_grow_tile(b, chunks: int) -> None:
    _check(load_library().qsgs_batch_set_grow_tile(b, chunks), "qsgs_batch_set_grow_tile")


def qsgs_batch_set_profiling(b, enable: bool) -> None:
    _check(load_library().qsgs_batch_set_profiling(b, int(enable)), "qsgs_batch_set_profiling")


def qsgs_batch_profile(b) -> dict:
    buf = (QsgsProfileEntry * 16)()
    n = _check(load_library().qsgs_batch_profile(b, buf, 16), "qsgs_batch_profile")
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(min(n, 16))}


def qsgs_batch_destroy(b) -> None:
    if b:
        load_library().qsgs_batch_destroy(b)


# ---- convenience wrapper ---------------------------------------------------
@dataclass
class Stats:
    solid_count: int
    target_count: int
    front_size: int
    n_candidates: int
    n_seeds: int
    sum_front: int
    steps: int
    status: int
    launches: int
    sum_draws: int


class Generator:
    """One realization bound to a torch-allocated workspace and stream."""

    def __init__(self, params: dict, device=None, stream=None, workspace=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libqsgs needs a CUDA device; there is no CPU fallback")
        load_library()
        self.params = dict(params)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.nbytes = qsgs_workspace_bytes(self.params)
        if self.nbytes == 0:
            raise QsgsError(QSGS_ERR_INVALID, "qsgs_workspace_bytes")
        with torch.cuda.device(self.device):
            if workspace is None:
                workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.workspace = workspace
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.handle = qsgs_create(self.params, workspace.data_ptr(), workspace.numel(),
                                      self.stream.cuda_stream)
        p = make_params(self.params)
        self.shape = (p.nz, p.ny, p.nx)
        self.n = p.nx * p.ny * p.nz
        self.words = ((p.nx + 31) // 32) * p.ny * p.nz

    def seed(self) -> None:
        qsgs_seed(self.handle)

    def grow(self, max_steps: int = 0) -> Stats:
        _, s = qsgs_grow_until(self.handle, max_steps)
        return Stats(**s)

    def query(self) -> Stats:
        return Stats(**qsgs_query(self.handle))

    def fetch(self, out=None, fmt: str = "u8"):
        """Phase map as a uint8 (nz, ny, nx) tensor, or the packed uint32
        words (fmt='packed').  ``out`` may be a CUDA or CPU tensor; a pinned
        CPU tensor is written by the device directly."""
        import torch
        f = QSGS_FMT_U8 if fmt == "u8" else QSGS_FMT_PACKED
        if out is None:
            if f == QSGS_FMT_U8:
                out = torch.empty(self.shape, dtype=torch.uint8, device=self.device)
            else:
                out = torch.empty(self.words, dtype=torch.int32, device=self.device)
        dst = (QSGS_DST_DEVICE if out.is_cuda else
               QSGS_DST_HOST_MAPPED if out.is_pinned() else QSGS_DST_HOST)
        qsgs_fetch(self.handle, out.data_ptr(), out.numel() * out.element_size(), f, dst)
        return out

    def snapshot(self, out=None):
        """The realization's state between growth calls, as a uint8 tensor
        (pinned host memory by default; ``out`` may be any CPU or CUDA
        uint8 tensor of at least ``qsgs_snapshot_bytes`` bytes)."""
        import torch
        n = qsgs_snapshot_bytes(self.params)
        if out is None:
            out = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        kind = QSGS_DST_DEVICE if out.is_cuda else QSGS_DST_HOST
        qsgs_snapshot(self.handle, out.data_ptr(), out.numel() * out.element_size(), kind)
        return out

    def restore(self, snap) -> None:
        """Continues the realization saved in ``snap`` (a tensor written by
        ``snapshot`` of a generator with the same parameters)."""
        kind = QSGS_DST_DEVICE if snap.is_cuda else QSGS_DST_HOST
        qsgs_restore(self.handle, snap.data_ptr(), snap.numel() * snap.element_size(), kind)

    def set_profiling(self, enable: bool = True) -> None:
        qsgs_set_profiling(self.handle, enable)

    def profile(self) -> dict:
        return qsgs_profile(self.handle)

    def set_grow_blocks(self, blocks: int) -> None:
        qsgs_set_grow_blocks(self.handle, blocks)

    def set_grow_tile(self, chunks: int) -> None:
        qsgs_set_grow_tile(self.handle, chunks)

    def set_mode(self, mode: int) -> None:
        """QSGS_MODE_LIETS (default) or QSGS_MODE_FULLFIELD (comparator)."""
        qsgs_set_mode(self.handle, mode)

    def set_blocked(self, blocked) -> None:
        """Packed int32 device tensor of the cells of earlier phases (kept
        referenced here while the handle uses it), or None."""
        self._blocked = blocked
        qsgs_set_blocked(self.handle, 0 if blocked is None else blocked.data_ptr())

    def set_interaction(self, labels, probs) -> None:
        """Interacting phase (R13): `labels` is the uint8 device map of the
        earlier phases (0 = unassigned), `probs` maps a label m to its
        (I_face, I_edge, I_corner) (a dict, or rows for m = 1, 2, ...); the
        phase also grows into those cells.  None clears it."""
        import torch
        if labels is None:
            self._labels = self._inter_scratch = None
            qsgs_set_interaction(self.handle, 0, [], 0, 0)
            return
        if isinstance(probs, dict):
            n = max(probs) if probs else 0
            rows = [tuple(probs.get(m, (0.0, 0.0, 0.0))) for m in range(1, n + 1)]
        else:
            rows = [tuple(r) for r in probs]
        nbytes = qsgs_interaction_bytes(self.params)
        with torch.cuda.device(self.device):
            scratch = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)  # the labels may come from torch's stream
        self._labels, self._inter_scratch = labels, scratch
        qsgs_set_interaction(self.handle, labels.data_ptr(), rows, scratch.data_ptr(), nbytes)

    def fetch_label(self, labels, label: int) -> None:
        """Writes `label` into the uint8 device map `labels` at this phase's cells."""
        qsgs_fetch_label(self.handle, labels.data_ptr(), labels.numel(), label)

    def fetch_or(self, blocked) -> None:
        """ORs this phase's cells into the packed int32 device tensor `blocked`."""
        qsgs_fetch_or(self.handle, blocked.data_ptr(), blocked.numel() * 4)

    def time_grow(self, grow_blocks: int = 0, reps: int = 5) -> float:
        return qsgs_time_grow(self.handle, grow_blocks, reps)

    def close(self) -> None:
        if getattr(self, "handle", None):
            qsgs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def word_count(params: dict) -> int:
    """Occupancy-grid words of a realization, rounded up to 32 (its share
    of a batch word space)."""
    p = make_params(params)
    words = ((p.nx + 31) // 32) * p.ny * p.nz
    return (words + 31) // 32 * 32


class Batch:
    """Many realizations advanced by the same launches (see qsgs.h)."""

    def __init__(self, max_members: int, max_words: int, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libqsgs needs a CUDA device; there is no CPU fallback")
        load_library()
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.nbytes = qsgs_batch_workspace_bytes(max_members, max_words)
        if self.nbytes == 0:
            raise QsgsError(QSGS_ERR_INVALID, "qsgs_batch_workspace_bytes")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.handle = qsgs_batch_create(max_members, max_words, self.workspace.data_ptr(),
                                            self.nbytes, self.stream.cuda_stream)
        self.members: list[Generator] = []

    def set_members(self, generators) -> None:
        self.members = list(generators)
        qsgs_batch_set_members(self.handle, [g.handle for g in self.members])

    def seed(self) -> None:
        qsgs_batch_seed(self.handle)

    def advance(self, max_steps: int = 0) -> None:
        qsgs_batch_advance(self.handle, max_steps)

    def query(self) -> list[Stats]:
        return [Stats(**d) for d in qsgs_batch_query(self.handle, len(self.members))]

    def run(self, max_steps: int = 0) -> list[Stats]:
        self.seed()
        self.advance(max_steps)
        return self.query()

    def set_grow_blocks(self, blocks: int) -> None:
        qsgs_batch_set_grow_blocks(self.handle, blocks)

    def set_grow_tile(self, chunks: int) -> None:
        qsgs_batch_set_grow_tile(self.handle, chunks)

    def set_profiling(self, enable: bool = True) -> None:
        qsgs_batch_set_profiling(self.handle, enable)

    def profile(self) -> dict:
        return qsgs_batch_profile(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            qsgs_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(params: dict, device=None, fmt: str = "u8"):
    """Seed and grow one realization; returns (phase tensor on the device, Stats)."""
    g = Generator(params, device=device)
    try:
        g.seed()
        st = g.grow()
        out = g.fetch(fmt=fmt)
        return out, st
    finally:
        g.close()


def generate_phases(phases: list, device=None, interactions=None):
    """Sec. 2.1 steps 4-5: phase k (k = 1, 2, ...) grows on the cells no
    earlier phase holds -- and, when interactions[k - 1] is a dict {m:
    (I_face, I_edge, I_corner)}, also into cells of the earlier phases m
    (R13), which become phase k's.  Returns the uint8 label map (nz, ny, nx)
    on the device (0 = matrix) and every phase's Stats.  All phases must
    have the same grid dims and domain kind."""
    import torch
    if not phases or len(phases) > 255:
        raise ValueError("1 .. 255 phases")
    first = make_params(phases[0])
    dims = (first.nx, first.ny, first.nz, first.periodic)
    dev = torch.device(device) if device is not None else torch.device(
        "cuda", torch.cuda.current_device())
    words = word_count(phases[0])
    blocked = torch.zeros(words, dtype=torch.int32, device=dev)
    labels = torch.zeros((first.nz, first.ny, first.nx), dtype=torch.uint8, device=dev)
    torch.cuda.synchronize(dev)  # the zero fills ran on torch's stream
    stats = []
    for k, p in enumerate(phases, start=1):
        q = make_params(p)
        if (q.nx, q.ny, q.nz, q.periodic) != dims:
            raise ValueError("all phases need the same grid")
        g = Generator(p, device=dev)
        spec = interactions[k - 1] if interactions else None
        try:
            if spec:
                if any(not 1 <= m < k for m in spec):
                    raise ValueError(f"phase {k} can only enter earlier phases")
                g.set_interaction(labels, spec)
            else:
                g.set_blocked(blocked if k > 1 else None)
            g.seed()
            stats.append(g.grow())
            g.fetch_label(labels, k)
            g.fetch_or(blocked)
        finally:
            g.close()
    return labels, stats
