"""qsgs_front_count_static: the front count on library-owned static scratch
(no allocation) must equal the front size the generator reports through
qsgs_query, call after call.  Collected last on purpose: it has to pass
after every other GPU test has used the library in the same process."""
import ctypes

import numpy as np
import pytest

from paper_2602_11734_gb300 import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def Q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_11734_gb300 import build, qsgs
    build.build()
    qsgs.load_library()
    return qsgs


def _count(Q, grid, p, stream=0):
    out = ctypes.c_uint64(12345)
    rc = Q.load_library().qsgs_front_count_static(ctypes.c_void_p(grid.data_ptr()), p["nx"], p["ny"],
                                                  p["nz"], ctypes.c_void_p(stream), ctypes.byref(out))
    return rc, out.value


@pytest.mark.parametrize("dims", [(72, 70, 68), (33, 40, 29), (130, 96, 101)])
def test_static_front_count_equals_query(oracle, Q, dims):
    nx, ny, nz = dims
    p = dict(workloads.small_64(), nx=nx, ny=ny, nz=nz, spacing_s=3, seed=nx + ny)
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow()
        grid = g.fetch(fmt="packed")
        torch.cuda.synchronize()
        first = _count(Q, grid, p, g.stream.cuda_stream)
        second = _count(Q, grid, p, g.stream.cuda_stream)
        assert first == (Q.QSGS_OK, st.front_size)
        assert second == (Q.QSGS_OK, st.front_size)
        assert st.front_size == oracle.run(p).front_size
    finally:
        g.close()


def test_static_front_count_mid_run_and_default_stream(Q):
    # Mid-run grids too (front of the current grid), on the legacy stream.
    p = dict(workloads.small_64(), nx=90, ny=64, nz=77, seed=9)
    g = Q.Generator(p)
    try:
        g.seed()
        g.grow(4)
        grid = g.fetch(fmt="packed")
        torch.cuda.synchronize()
        words = grid.cpu().numpy().view(np.uint32).reshape(p["nz"], p["ny"], -1)
        bits = np.unpackbits(words.view(np.uint8), bitorder="little").reshape(
            p["nz"], p["ny"], -1)[:, :, :p["nx"]].astype(bool)
        pad = np.pad(bits, 1, constant_values=True)  # outside the domain: not a void
        void_nb = np.zeros_like(bits)
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx or dy or dz:
                        void_nb |= ~pad[1 + dz:1 + dz + p["nz"], 1 + dy:1 + dy + p["ny"],
                                        1 + dx:1 + dx + p["nx"]]
        want = int((bits & void_nb).sum())
        assert _count(Q, grid, p) == (Q.QSGS_OK, want)
        assert _count(Q, grid, p) == (Q.QSGS_OK, want)
    finally:
        g.close()


# The stated limit of the static scratch: 16,707,584 words.  A grid of
# 32 x 4096 x 4079 voxels (one word per row) has exactly that many.
LIMIT_WORDS = 16_707_584


def test_static_front_count_at_its_word_limit(Q):
    # The largest grid the scratch serves: the count must use the tile
    # status words up to the end of the static array, and still equal the
    # front the generator reports, on two calls in a row; one plane more is
    # refused before the device is touched.
    p = dict(workloads.small_64(), nx=32, ny=4096, nz=4079, cd=0.002, seed=77)
    assert (p["nx"] + 31) // 32 * p["ny"] * p["nz"] == LIMIT_WORDS
    g = Q.Generator(p)
    try:
        g.seed()
        st = g.grow()
        assert st.status == Q.QSGS_OK
        grid = g.fetch(fmt="packed")
        torch.cuda.synchronize()
        assert grid.numel() == LIMIT_WORDS
        assert _count(Q, grid, p, g.stream.cuda_stream) == (Q.QSGS_OK, st.front_size)
        assert _count(Q, grid, p) == (Q.QSGS_OK, st.front_size)
        assert st.front_size > 0
        over = dict(p, nz=p["nz"] + 1)
        assert _count(Q, grid, over)[0] == Q.QSGS_ERR_WORKSPACE
    finally:
        g.close()


def test_static_front_count_rejects_oversized_grids(Q):
    small = torch.zeros(4, dtype=torch.int32, device="cuda")
    # 1024^3 needs 34,603,008 words: more than the static scratch serves.
    p = dict(nx=1024, ny=1024, nz=1024)
    assert _count(Q, small, p)[0] == Q.QSGS_ERR_WORKSPACE
    assert _count(Q, small, dict(nx=0, ny=4, nz=4))[0] == Q.QSGS_ERR_INVALID
