"""Pins of the oracle's base generators and output conversions (CPU only).

Each test checks the oracle against something other than itself: a value fixed
by the C++ standard, a library implementation of the same generator (Python's
``random``, numpy's ``MT19937``, libstdc++'s ``std::mt19937[_64]``), or an
invariant that a wrong constant, shift or index would break.
"""
import os
import random

import numpy as np
import pytest

import oracle as O
from conftest import ROOT, run_stdmt
from paper_2309_16682_gb300 import inputs as I




def _golden_10000th():
    rows = {}
    with open(os.path.join(ROOT, "tests", "golden", "cxx_standard_10000th.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v, seed, idx, val = line.split()
            rows[v] = (int(seed), int(idx), int(val))
    return rows


@pytest.mark.parametrize("name,variant", [("mt32", O.MT32), ("mt64", O.MT64)])
def test_cxx_standard_10000th(name, variant):
    seed, idx, val = _golden_10000th()[name]
    z = O.outputs(O.seed_state(variant, seed), idx)
    assert int(z[idx - 1]) == val


def test_mt32_matches_python_random_from_arbitrary_state():
    """Python's random module is MT19937-32; setstate() accepts any 624 words."""
    rng = np.random.default_rng(11)
    for trial in range(3):
        words = rng.integers(0, 2**32, size=624, dtype=np.uint64)
        r = random.Random()
        r.setstate((3, tuple(int(w) for w in words) + (624,), None))
        ref = [r.getrandbits(32) for _ in range(3000)]
        st = O.State(O.MT32, words.astype(np.uint32), 0)
        got = O.outputs(st, 3000)
        assert [int(x) for x in got] == ref


@pytest.mark.parametrize("seed", [0, 1, 5489, 2**32 - 1, 123456789])
def test_mt32_matches_numpy_legacy_seeding(seed):
    bg = np.random.MT19937()
    bg._legacy_seeding(seed)
    ref = bg.random_raw(2000)
    got = O.outputs(O.seed_state(O.MT32, seed), 2000)
    assert np.array_equal(got.astype(np.uint64), ref)


@pytest.mark.parametrize("seed", [0, 5489, 2**64 - 1, 0x0123456789ABCDEF])
def test_mt64_matches_libstdcxx(stdmt, seed):
    ref = run_stdmt(stdmt, 64, seed, 0, 1500)
    got = O.outputs(O.seed_state(O.MT64, seed), 1500)
    assert [int(x) for x in got] == ref


@pytest.mark.parametrize("seed", [1, 5489, 2**32 - 1])
def test_mt32_matches_libstdcxx(stdmt, seed):
    ref = run_stdmt(stdmt, 32, seed, 0, 1500)
    got = O.outputs(O.seed_state(O.MT32, seed), 1500)
    assert [int(x) for x in got] == ref


def test_f32_conversion_matches_numpy_generator():
    """numpy's Generator.random(dtype=float32) on an MT19937 bit generator is
    (next_uint32 >> 8) * 2^-24: the library form of the f32 reading."""
    bg = np.random.MT19937()
    bg._legacy_seeding(42)
    ref = np.random.Generator(bg).random(5000, dtype=np.float32)
    w = O.outputs(O.seed_state(O.MT32, 42), 5000)
    assert np.array_equal(O.convert(O.MT32, w, "f32"), ref)


def test_f64_pair_conversion_matches_python_random():
    """Python's random.random() is the 53-bit double built from two MT19937-32
    words, (a >> 5) * 2^26 + (b >> 6), scaled by 2^-53."""
    rng = np.random.default_rng(3)
    words = rng.integers(0, 2**32, size=624, dtype=np.uint64)
    r = random.Random()
    r.setstate((3, tuple(int(w) for w in words) + (624,), None))
    ref = np.array([r.random() for _ in range(2000)])
    w = O.outputs(O.State(O.MT32, words.astype(np.uint32), 0), 4000)
    assert np.array_equal(O.convert(O.MT32, w, "f64"), ref)


def test_u64_pair_conversion_is_little_endian_view():
    w = O.outputs(O.seed_state(O.MT32, 7), 1000)
    assert np.array_equal(O.convert(O.MT32, w, "u64"), w.view("<u8").astype(np.uint64))


def test_mt64_float_conversions_invariants():
    w = O.outputs(O.seed_state(O.MT64, 9), 3000)
    f = O.convert(O.MT64, w, "f64")
    assert np.all((f >= 0) & (f < 1))
    assert np.array_equal((f * 2.0**53).astype(np.uint64), w >> np.uint64(11))
    g = O.convert(O.MT64, w, "f32")
    assert g.dtype == np.float32 and np.all((g >= 0) & (g < 1))
    assert np.array_equal((g.astype(np.float64) * 2.0**24).astype(np.uint64), w >> np.uint64(40))


def test_f32_endpoints():
    w = np.array([0, 0xFF, 0x100, 0xFFFFFFFF], dtype=np.uint32)
    f = O.convert(O.MT32, w, "f32")
    assert f[0] == 0.0 and f[1] == 0.0 and f[2] == np.float32(2.0**-24)
    assert f[3] == np.float32(1.0 - 2.0**-24) and f[3] < 1.0


def test_sfmt_certified_seeds_have_odd_parity():
    for s in [0, 1, 1234, 5489, 2**32 - 1]:
        assert O.sfmt_inner(O.seed_state(O.SFMT, s)) == 1


def _numpy_mt_key(seed):
    """The 624-word array numpy's own MT19937 holds right after its legacy
    integer seeding (the 32-bit initialisation that SFMT19937 also runs over
    its 624 sub-words, element k being sub-words 4k..4k+3)."""
    bg = np.random.MT19937()
    bg._legacy_seeding(seed)
    st = bg.state["state"]
    assert st["pos"] == 624
    return np.asarray(st["key"], dtype=np.uint32)


@pytest.mark.parametrize("seed", [0, 1, 1234, 5489, 2**31, 2**32 - 1])
def test_sfmt_seeding_is_numpy_mt_key_up_to_certification(seed):
    """Seeded SFMT buffer = numpy's MT19937 key array, except for the one bit
    that certification may flip: the parity vector's lowest set bit, sub-word 0
    bit 0.  The flip happens exactly when the key array fails the check."""
    key = _numpy_mt_key(seed)
    st = O.seed_state(O.SFMT, seed)
    assert st.k == 0
    diff = st.words ^ key
    assert np.count_nonzero(diff[1:]) == 0
    assert diff[0] in (0, 1)
    key_parity = O.sfmt_inner(O.State(O.SFMT, key, 0))
    assert diff[0] == (1 - key_parity)
    assert O.sfmt_inner(st) == 1


def test_sfmt_certification_flips_when_needed():
    """Over many seeds both outcomes occur (an even key array is fixed, an odd
    one is left alone), so the test above exercises both branches."""
    flipped = [int((O.seed_state(O.SFMT, s).words ^ _numpy_mt_key(s))[0]) for s in range(64)]
    assert 0 < sum(flipped) < 64


def test_sfmt_64bit_seed_taken_mod_2_32():
    for s in [7, 2**32 - 1]:
        assert np.array_equal(O.seed_state(O.SFMT, s + (5 << 32)).words, O.seed_state(O.SFMT, s).words)


def test_splitmix64_two_forms_and_published_first_value():
    assert I.splitmix64_scalar(0, 1)[0] == 0xE220A8397B1DCDAF
    for s in [0, 1, 2, 2**64 - 1, 0xDEADBEEF]:
        assert [int(x) for x in I.splitmix64(s, 64)] == I.splitmix64_scalar(s, 64)
