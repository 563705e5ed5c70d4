"""Out-of-bounds write checks (GPU), in place of a memory sanitizer.

Every output is written into a view in the middle of a larger device buffer
whose guard regions hold a canary pattern; after the call the guards must be
untouched and the view must hold the same values as an unguarded call (which
the parity tests tie to the oracle).  Sizes are chosen to hit partial vectors,
partial blocks, odd word offsets, one-element and single-lane cases.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GUARD = 4096          # elements on each side
CANARY = 0x5A


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    m.lib()
    return m


def _guarded(vmt, shape, dtype, shift=0):
    """(view, whole, element size, elements) -- a view of `shape` inside a
    canary-filled byte buffer, starting `shift` elements past the guard (so
    that shift = 1 gives an output that is not 16-byte aligned)."""
    tdt = vmt._torch_dtype(dtype)
    esize = torch.empty(0, dtype=tdt).element_size()
    n = int(np.prod(shape)) if shape else 0
    whole = torch.full(((n + 2 * GUARD) * esize,), CANARY, dtype=torch.uint8, device="cuda")
    lo = (GUARD + shift) * esize
    view = whole[lo:lo + n * esize].view(tdt)
    return view.view(*shape) if shape else view, whole, esize, (n, shift)


def _check_guards(whole, esize, ns):
    n, shift = ns if isinstance(ns, tuple) else (ns, 0)
    torch.cuda.synchronize()
    lo = whole[:(GUARD + shift) * esize]
    hi = whole[(GUARD + shift + n) * esize:]
    assert bool((lo == CANARY).all()), "write below the output"
    assert bool((hi == CANARY).all()), "write above the output"


def _same(a, b):
    return torch.equal(a.view(torch.uint8), b.contiguous().view(torch.uint8))


CASES = [("mt32", 1, "u32"), ("mt32", 2, "u64"), ("mt32", 4, "f64"), ("mt32", 16, "f32"),
         ("mt64", 1, "f64"), ("mt64", 8, "f32"), ("mt64", 16, "u64"),
         ("sfmt", 1, "u32"), ("sfmt", 4, "f64"), ("sfmt", 16, "f32")]


@pytest.mark.parametrize("variant,M,dtype", CASES)
def test_lockstep_calls_stay_in_bounds(vmt, variant, M, dtype):
    count = 5
    ref = vmt.VGenerator(variant, M, list(range(1, count + 1)))
    g = vmt.VGenerator(variant, M, list(range(1, count + 1)))
    for n, shift in [(1, 0), (3, 1), (M * 624 - 1, 0), (2 * M * 624 + 5, 1), (7777, 0), (4096, 1)]:
        view, whole, esize, tot = _guarded(vmt, (count, n), dtype, shift)
        g.generate(n, dtype, out=view)
        _check_guards(whole, esize, tot)
        assert _same(view, ref.generate(n, dtype)), (variant, M, dtype, n, shift)


@pytest.mark.parametrize("variant,M", [("mt32", 16), ("mt64", 8), ("sfmt", 4)])
def test_fused_segments_stay_in_bounds(vmt, variant, M):
    native = "u64" if variant == "mt64" else "u32"
    flt = "f64" if variant == "mt64" else "f32"
    segs = [(1001, native), (333, flt)]
    count = 3
    g = vmt.VGenerator(variant, M, [9, 8, 7])
    ref = vmt.VGenerator(variant, M, [9, 8, 7])
    bufs = [_guarded(vmt, (count, n), dt) for n, dt in segs]
    g.generate_multi(segs, outs=[b[0] for b in bufs])
    for (n, dt), (view, whole, esize, tot) in zip(segs, bufs):
        _check_guards(whole, esize, tot)
        assert _same(view, ref.generate(n, dt))


@pytest.mark.parametrize("variant,M,dtype", [("mt32", 4, "u32"), ("mt32", 1, "f32"), ("mt64", 2, "u64"),
                                             ("sfmt", 8, "u32")])
def test_ragged_calls_stay_in_bounds(vmt, variant, M, dtype):
    lens = [0, 1, 2, 624 * M + 3, 5000, 17]
    g = vmt.VGenerator(variant, M, list(range(40, 40 + len(lens))))
    bufs = [_guarded(vmt, (n,), dtype) for n in lens]
    g.generate_ragged(lens, dtype, outs=[b[0] for b in bufs])
    for k, (n, (view, whole, esize, tot)) in enumerate(zip(lens, bufs)):
        _check_guards(whole, esize, tot)
        alone = vmt.VGenerator(variant, M, [40 + k]).generate(n, dtype)[0]
        assert _same(view, alone), (variant, M, dtype, n)


@pytest.mark.parametrize("variant,dtype,n", [("mt32", "u32", 1), ("mt32", "f32", 1_000_001), ("mt64", "u64", 77_777),
                                             ("sfmt", "u32", 2_000_003)])
def test_single_stream_stays_in_bounds(vmt, variant, dtype, n):
    view, whole, esize, tot = _guarded(vmt, (n,), dtype)
    vmt.stream_generate(variant, 3, n, dtype, out=view)
    _check_guards(whole, esize, tot)
    assert _same(view, vmt.stream_generate(variant, 3, n, dtype))
