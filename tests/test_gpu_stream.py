"""Exact single-stream mode (GPU): one base generator's stream produced in
parallel chunks equals the library routine (std::mt19937, std::mt19937_64)
and the oracle, across chunk boundaries, with and without a start offset."""
import numpy as np
import pytest

import oracle as O
from conftest import run_stdmt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    m.lib()
    return m


def _np(t):
    if t.dtype == torch.uint32:
        return t.cpu().view(torch.int32).numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.cpu().view(torch.int64).numpy().view(np.uint64)
    return t.cpu().numpy()


def _windows(n, chunk):
    """(start, length) windows at the start, around every chunk boundary
    among the first few, and at the end."""
    w = [(0, 700)]
    for j in range(1, min(4, n // chunk) + 1):
        w.append((max(0, j * chunk - 300), 600))
    w.append((n - 500, 500))
    return [(a, min(b, n - a)) for a, b in w if a < n]


@pytest.mark.parametrize("bits,seed,skip", [(32, 5489, 0), (32, 12345, 777), (64, 5489, 0), (64, 42, 1001)])
def test_stream_equals_std_engine(vmt, stdmt, bits, seed, skip):
    variant, dtype = ("mt32", "u32") if bits == 32 else ("mt64", "u64")
    n = 3_000_001
    got = _np(vmt.stream_generate(variant, seed, n, dtype, jump=skip))
    words = 624 if bits == 32 else 312
    chunk = max(64, -(-(-(-n // words)) // 2048)) * words
    for a, L in _windows(n, chunk):
        ref = np.array(run_stdmt(stdmt, bits, seed, skip + a, L), dtype=np.uint32 if bits == 32 else np.uint64)
        assert np.array_equal(got[a:a + L], ref), (bits, seed, skip, a)


@pytest.mark.parametrize("variant,dtype", [("sfmt", "u32"), ("sfmt", "f32"), ("mt32", "f32"), ("mt64", "f64")])
def test_stream_matches_oracle(vmt, oracle_polys, variant, dtype):
    v = O.VARIANTS[variant]
    n, seed, d = 1_000_003, 99, 123456789
    got = _np(vmt.stream_generate(variant, seed, n, dtype, jump=d))
    words = {"mt32": 624, "mt64": 312, "sfmt": 624}[variant]
    chunk = max(64, -(-(-(-n // words)) // 2048)) * words
    lanes = O.lane_states(v, 1, seed, d)
    for a, L in _windows(n, chunk):
        ref = O.vstream(v, 1, seed, L, dtype, start_word=a, lanes=lanes)
        assert np.array_equal(got[a:a + L], ref), (variant, dtype, a)


def test_stream_long_fills_many_chunks(vmt, stdmt):
    n = 1 << 28   # 1 GiB of u32: 2048 chunks
    got = _np(vmt.stream_generate("mt32", 7, n, "u32"))
    for a in (0, n // 3, n - 1000):
        ref = np.array(run_stdmt(stdmt, 32, 7, a, 1000), dtype=np.uint32)
        assert np.array_equal(got[a:a + 1000], ref), a


def test_stream_rejects_bad_arguments(vmt):
    with pytest.raises(vmt.VMTError):
        vmt.stream_generate("mt64", 1, 10, "u32")
    assert vmt.stream_generate("mt32", 1, 0, "u32").numel() == 0
