"""The library's host polynomial helpers on an F2-linear generator other than
the three it ships kernels for (CPU).

The jump of Sec. 3.1 needs only the minimal polynomial of the transition on
the state's orbit, found by Berlekamp-Massey from output bits, and x^J modulo
it; nothing in that is specific to MT19937 or SFMT19937.  Here the C ABI's
vmt_poly_minpoly, vmt_poly_x2pow and vmt_poly_mulmod jump the 80-bit twisted
GFSR analogue of the matrix cross-check, and the result must equal the 80 x 80
transition matrix raised to J (a route that shares nothing with either
polynomial code).

Like MT19937's, the analogue's transition is singular: the low r bits of the
oldest word never reach an output, so the polynomial found from output bits
lacks the factor x that the freshly drawn state would need.  Every state from
the first step on lies in the image of the transition, where it suffices; the
start state is therefore taken one step after the random one.
"""
import numpy as np
import pytest

import test_oracle_matrix_jump as A

vmt = pytest.importorskip("paper_2309_16682_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_2309_16682_gb300 import build
    build.build()
    return vmt.lib()


def _orbit_bits(x0, bit, length):
    """Bit `bit` of the newest word, one per step of the analogue."""
    out, x = [], x0
    for _ in range(length):
        x = A.step(x)
        out.append((x[-1] >> bit) & 1)
    return np.array(out, np.uint8)


def _to_int(words):
    return sum(int(w) << (64 * i) for i, w in enumerate(words))


def _library_minpoly(x0):
    """Berlekamp-Massey (library) on each output bit until the polynomial
    annihilates the state itself, i.e. is the minimal polynomial on its orbit."""
    for bit in range(A.W):
        d, mu = vmt.poly_minpoly(_orbit_bits(x0, bit, 3 * A.DIM))
        mu = mu[:d // 64 + 1].copy()
        if A.horner(_to_int(mu), x0) == [0] * A.N:
            return d, mu
    raise AssertionError("no output bit reaches the minimal polynomial")


def _library_xpow(J, mu):
    chain = vmt.poly_x2pow(mu, 0, J.bit_length())
    acc = np.zeros(mu.size, np.uint64)
    acc[0] = 1
    for q in range(J.bit_length()):
        if (J >> q) & 1:
            acc = vmt.poly_mulmod(acc, chain[q], mu)
    return _to_int(acc)


@pytest.fixture(scope="module")
def analogue(lib):
    rng = np.random.default_rng(16682)
    x0 = A.step([int(v) for v in rng.integers(0, 1 << A.W, size=A.N)])
    d, mu = _library_minpoly(x0)
    return A.transition_matrix(), x0, d, mu


def test_library_minpoly_is_the_oracles(analogue):
    F, x0, d, mu = analogue
    ref = A.minimal_polynomial(x0)
    assert d == ref.bit_length() - 1 <= A.DIM
    assert _to_int(mu) == ref


@pytest.mark.parametrize("J", [1, 79, 80, 4097, 2**40 + 12345, 2**63 - 1, 3**50])
def test_library_jump_equals_matrix_power(analogue, J):
    F, x0, d, mu = analogue
    if J < 5000:
        brute = x0
        for _ in range(J):
            brute = A.step(brute)
    else:
        brute = A.from_bits(A.matpow2(F, J) @ A.to_bits(x0) % 2)
    assert A.horner(_library_xpow(J, mu), x0) == brute
