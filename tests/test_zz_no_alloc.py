"""vmt_jump_noalloc against vmt_jump (GPU).

vmt_jump_noalloc exists for callers that cannot allocate device memory (a
framework's caching allocator owning the free HBM, allocation-free real-time
loops, plug-ins whose host forbids library allocations).  It must give exactly
what vmt_jump gives.  Two identical generator sets are jumped, one with each
entry point, twice in a row with different polynomials; the outputs generated
after each jump must agree bit for bit (the tests' tolerance for integer
output is zero).  Further cases: a call at exactly the static limit of
lane-states, one lane-state beyond it, and a polynomial in pinned host memory
that the caller overwrites as soon as the call returns.  The file is collected
last and needs nothing from the other test files, so it passes alone in a
fresh process and after the full suite.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMIT = 16384   # VMT_NOALLOC_MAX_LANE_STATES


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    L = m.lib()
    L.vmt_jump_noalloc.restype = ctypes.c_int
    L.vmt_jump_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    return m


def _u32(t):
    return t.cpu().view(torch.int32).numpy().view(np.uint32)


def _noalloc_jump_ptr(vmt, g, ptr, nbits):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = vmt.lib().vmt_jump_noalloc(g._h, ctypes.c_void_p(ptr), int(nbits), s)
    if rc != 0:
        raise vmt.VMTError(rc, vmt.lib().vmt_last_error().decode())


def _noalloc_jump(vmt, g, poly, nbits):
    poly = np.ascontiguousarray(poly, dtype=np.uint64)
    _noalloc_jump_ptr(vmt, g, poly.ctypes.data, nbits)


@pytest.mark.parametrize("variant,lanes", [("mt32", 16), ("sfmt", 4)])
def test_noalloc_jump_matches_jump_twice(vmt, variant, lanes):
    seeds = np.arange(1, 65, dtype=np.uint64) * np.uint64(2654435761)
    a = vmt.VGenerator(variant, lanes, seeds)
    b = vmt.VGenerator(variant, lanes, seeds)
    _ = a.generate(1001, "u32")
    _ = b.generate(1001, "u32")
    for d, trim in [(123456789, 0), (2**63 + 12345, 37)]:
        p = vmt.jump_poly(variant, d)
        nbits = p.size * 64 - trim          # second call: nbits not a multiple of 64
        a.jump(p, nbits)
        _noalloc_jump(vmt, b, p, nbits)
        ra = _u32(a.generate(7000, "u32"))
        rb = _u32(b.generate(7000, "u32"))
        assert np.array_equal(ra, rb)


def test_noalloc_at_the_limit_twice(vmt):
    # 1024 generators x 16 lanes = exactly the largest accepted call: the last
    # work item sits at the end of the static array
    seeds = np.arange(7, 7 + 1024, dtype=np.uint64)
    a = vmt.VGenerator("mt32", 16, seeds)
    b = vmt.VGenerator("mt32", 16, seeds)
    assert 1024 * 16 == LIMIT
    for d in (987654321, 2**40 + 3):
        p = vmt.jump_poly("mt32", d)
        a.jump(p, p.size * 64)
        _noalloc_jump(vmt, b, p, p.size * 64)
        ra = _u32(a.generate(16 * 640, "u32"))
        rb = _u32(b.generate(16 * 640, "u32"))
        assert np.array_equal(ra, rb)


def test_noalloc_pinned_poly_overwritten_after_the_call(vmt):
    seeds = np.arange(100, 132, dtype=np.uint64)
    a = vmt.VGenerator("mt64", 8, seeds)
    b = vmt.VGenerator("mt64", 8, seeds)
    p = vmt.jump_poly("mt64", 2**50 + 99)
    pinned = torch.empty(p.size, dtype=torch.int64, pin_memory=True)
    pinned.numpy().view(np.uint64)[:] = p
    _ = a.generate(1 << 22, "u64")
    a.jump(p, p.size * 64)
    # queue work ahead of the call on the same stream, so that anything still
    # reading the host buffer asynchronously would read it after the overwrite
    _ = b.generate(1 << 22, "u64")
    _noalloc_jump_ptr(vmt, b, pinned.data_ptr(), p.size * 64)
    pinned.fill_(-1)                      # the caller reuses its buffer at once
    ra = a.generate(8 * 1000, "u64").cpu().numpy()
    rb = b.generate(8 * 1000, "u64").cpu().numpy()
    assert np.array_equal(ra, rb)


def test_noalloc_rejects_states_beyond_the_limit(vmt):
    g = vmt.VGenerator("mt32", 16, np.arange(1100, dtype=np.uint64))   # 17600 lane-states
    p = vmt.jump_poly("mt32", 5)
    with pytest.raises(vmt.VMTError) as ei:
        _noalloc_jump(vmt, g, p, p.size * 64)
    assert ei.value.code == vmt.VMT_EINVAL
    assert "VMT_NOALLOC_MAX_LANE_STATES" in str(ei.value)
    g1 = vmt.VGenerator("mt32", 1, np.arange(LIMIT + 1, dtype=np.uint64))   # one lane-state too many
    with pytest.raises(vmt.VMTError) as ei:
        _noalloc_jump(vmt, g1, p, p.size * 64)
    assert ei.value.code == vmt.VMT_EINVAL
