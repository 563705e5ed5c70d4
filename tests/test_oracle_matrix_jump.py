"""Matrix-form jump-ahead as an independent cross-check of the polynomial form.

Sec. 3.1 describes two routes to a jumped state: the matrix B = F^J applied to
X, and the polynomial c(F) X with c = x^J mod the characteristic polynomial.
For MT19937 the matrix route is out of reach (a 19937 x 19937 bit matrix
raised to J = 2^19933), so it is checked here on a small analogue with the
same structure as eq. step -- a twisted GFSR with w = 16, n = 5, m = 2, r = 7
and an arbitrary twist constant -- whose 80 x 80 transition matrix can be
powered directly.  The polynomial route uses the oracle's own routines
(Berlekamp-Massey, modular products); the matrix route shares nothing with
them.  Both must agree with each other for huge J and with plain stepping for
small J.
"""
import numpy as np
import pytest

import oracle as O

W, N, MM, R, A = 16, 5, 2, 7, 0xB4F1
LOWER = (1 << R) - 1
UPPER = ((1 << W) - 1) ^ LOWER
DIM = N * W


def step(x):
    """One step of the analogue on the window (x_i .. x_{i+n-1}), eq. step."""
    y = (x[0] & UPPER) | (x[1] & LOWER)
    new = x[MM] ^ (y >> 1) ^ (A if y & 1 else 0)
    return x[1:] + [new]


def to_bits(x):
    return np.array([(x[i] >> b) & 1 for i in range(N) for b in range(W)], dtype=np.uint8)


def from_bits(v):
    return [int(sum(int(v[i * W + b]) << b for b in range(W))) for i in range(N)]


def transition_matrix():
    """Column j = F applied to the j-th unit state."""
    F = np.zeros((DIM, DIM), dtype=np.uint8)
    for j in range(DIM):
        e = np.zeros(DIM, np.uint8)
        e[j] = 1
        F[:, j] = to_bits(step(from_bits(e)))
    return F


def matmul2(a, b):
    return (a.astype(np.int64) @ b.astype(np.int64) % 2).astype(np.uint8)


def matpow2(F, e):
    out = np.eye(DIM, dtype=np.uint8)
    base = F.copy()
    while e:
        if e & 1:
            out = matmul2(out, base)
        e >>= 1
        if e:
            base = matmul2(base, base)
    return out


def minimal_polynomial(x0):
    """lcm over all state bits of the Berlekamp-Massey polynomials of the
    sequence X, F X, F^2 X, ... (the minimal polynomial of F on X's orbit)."""
    seq = [x0]
    for _ in range(3 * DIM):
        seq.append(step(seq[-1]))
    bits = np.array([to_bits(s) for s in seq])          # [time][bit]
    mu = 1
    for b in range(DIM):
        L, m = O.berlekamp_massey(bits[:, b])
        mb = O.to_int(m)
        if mb.bit_length() - 1 != L:
            continue
        mu = O._gf2_div(O._gf2_mul(mu, mb), O._gf2_gcd(mu, mb))
    return mu


def xpow_mod(e, mu):
    """x^e mod mu by square and multiply with the oracle's modular product."""
    m = O.from_int(mu)
    acc = O.from_int(1)
    base = O.poly_mod(O.from_int(2), m)
    while e:
        if e & 1:
            acc = O.poly_mulmod(acc, base, m)
        e >>= 1
        if e:
            base = O.poly_mulmod(base, base, m)
    return O.to_int(acc)


def horner(c, x0):
    """c(F) X: acc <- F(acc) xor c_i X from the top coefficient down."""
    acc = [0] * N
    for i in range(c.bit_length() - 1, -1, -1):
        acc = step(acc)
        if (c >> i) & 1:
            acc = [a ^ b for a, b in zip(acc, x0)]
    return acc


@pytest.fixture(scope="module")
def setup():
    rng = np.random.default_rng(2309)
    x0 = [int(v) for v in rng.integers(0, 1 << W, size=N)]
    return transition_matrix(), x0, minimal_polynomial(x0)


def test_minimal_polynomial_annihilates_the_orbit(setup):
    F, x0, mu = setup
    assert 1 < mu.bit_length() - 1 <= DIM
    assert horner(mu, x0) == [0] * N


@pytest.mark.parametrize("J", [1, 2, 7, 80, 81, 1000, 4097])
def test_small_jumps_three_ways(setup, J):
    F, x0, mu = setup
    brute = x0
    for _ in range(J):
        brute = step(brute)
    matrix = from_bits(matpow2(F, J) @ to_bits(x0) % 2)
    poly = horner(xpow_mod(J, mu), x0)
    assert matrix == brute and poly == brute


@pytest.mark.parametrize("J", [2**40 + 12345, 2**63 - 1, 3**50, 2**79])
def test_huge_jumps_matrix_equals_polynomial(setup, J):
    F, x0, mu = setup
    matrix = from_bits(matpow2(F, J) @ to_bits(x0) % 2)
    assert horner(xpow_mod(J, mu), x0) == matrix


def test_jumps_compose(setup):
    F, x0, mu = setup
    a, b = 2**33 + 5, 2**41 - 17
    ab = horner(xpow_mod(b, mu), horner(xpow_mod(a, mu), x0))
    assert ab == from_bits(matpow2(F, a + b) @ to_bits(x0) % 2)
