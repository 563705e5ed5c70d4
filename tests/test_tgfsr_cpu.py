"""The full-period twisted GFSR parameters in tests/golden/tgfsr_params.txt,
pinned without the polynomial routines that found them (CPU).

The stored parameters claim period 2^p - 1 for a generator of the shape of
eq. step (Sec. 2.1).  The check here uses only the transition matrix F over
GF(2) (dimension n w), built column by column from a plain Python step and
squared p times: F^(2^p) X = F X for a state X in the image of F (its orbit
has period dividing 2^p - 1, which is prime, so the period is exactly
2^p - 1 unless F X = X), and F X != X.  A wrong a, m or r, or a transposed
step, fails it.  The same matrix power also pins the polynomial route of the
library's host helpers for a huge jump.
"""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tgfsr_params.txt")


def load_params():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w, n, m, r, a, p = line.split()
        rows.append(dict(w=int(w), n=int(n), m=int(m), r=int(r), a=int(a, 16), p=int(p)))
    return rows


def step(x, g):
    lower = (1 << g["r"]) - 1
    upper = ((1 << g["w"]) - 1) ^ lower
    y = (x[0] & upper) | (x[1] & lower)
    return x[1:] + [x[g["m"]] ^ (y >> 1) ^ (g["a"] if y & 1 else 0)]


def to_bits(x, g):
    return np.array([(x[i] >> b) & 1 for i in range(g["n"]) for b in range(g["w"])], dtype=np.float64)


def from_bits(v, g):
    v = np.asarray(v).astype(np.int64) & 1
    return [int(sum(int(v[i * g["w"] + b]) << b for b in range(g["w"]))) for i in range(g["n"])]


def transition(g):
    dim = g["n"] * g["w"]
    F = np.zeros((dim, dim))
    for j in range(dim):
        e = np.zeros(dim)
        e[j] = 1
        F[:, j] = to_bits(step(from_bits(e, g), g), g)
    return F


def mat_pow2(F, e):
    """F^e over GF(2) (float products are exact: entries stay below 2^53)."""
    out = np.eye(F.shape[0])
    base = F.copy()
    while e:
        if e & 1:
            out = np.mod(out @ base, 2.0)
        e >>= 1
        if e:
            base = np.mod(base @ base, 2.0)
    return out


def image_state(g, seed):
    rng = np.random.default_rng(seed)
    return step([int(v) for v in rng.integers(0, 1 << g["w"], size=g["n"])], g)


@pytest.mark.parametrize("g", load_params(), ids=lambda g: f"p{g['p']}")
def test_stored_parameters_have_full_period(g):
    assert g["n"] * g["w"] - g["r"] == g["p"]
    F = transition(g)
    x = image_state(g, 2309 + g["p"])
    F2p = F.copy()
    for _ in range(g["p"]):
        F2p = np.mod(F2p @ F2p, 2.0)                   # F^(2^p)
    v = to_bits(x, g)
    assert from_bits(F2p @ v, g) == step(x, g)        # F^(2^p) X = F X: period divides 2^p - 1
    assert step(x, g) != x                            # and is not 1


@pytest.mark.parametrize("g", load_params(), ids=lambda g: f"p{g['p']}")
def test_library_polynomial_jump_equals_matrix_power(g):
    vmt = pytest.importorskip("paper_2309_16682_gb300")
    from paper_2309_16682_gb300 import build
    build.build()
    x = image_state(g, 77 + g["p"])
    # minimal polynomial from output bits (library Berlekamp-Massey)
    bits, y = [], x
    for _ in range(3 * g["p"]):
        y = step(y, g)
        bits.append(y[-1] & 1)
    d, mu = vmt.poly_minpoly(np.array(bits, np.uint8))
    assert d == g["p"]
    mu = mu[:d // 64 + 1].copy()
    J = 2**100 + 12345
    chain = vmt.poly_x2pow(mu, 0, J.bit_length())
    acc = np.zeros(mu.size, np.uint64)
    acc[0] = 1
    for q in range(J.bit_length()):
        if (J >> q) & 1:
            acc = vmt.poly_mulmod(acc, chain[q], mu)
    c = sum(int(wd) << (64 * i) for i, wd in enumerate(acc))
    # Horner: c(F) X
    h = [0] * g["n"]
    for i in range(c.bit_length() - 1, -1, -1):
        h = step(h, g)
        if (c >> i) & 1:
            h = [u ^ v for u, v in zip(h, x)]
    assert h == from_bits(mat_pow2(transition(g), J) @ to_bits(x, g), g)
