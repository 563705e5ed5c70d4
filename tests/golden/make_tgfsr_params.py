"""Writes tests/golden/tgfsr_params.txt: twisted GFSR parameters of full
period, found by search with the oracle's routines only.

A twisted GFSR of the shape of eq. step (Sec. 2.1) with w-bit words, n words
of state, middle distance m, separation point r and twist constant a moves
its state on p = n w - r effective bits (the low r bits of the oldest word
never reach an output).  Its period is 2^p - 1 exactly when the minimal
polynomial mu of its output sequence has degree p and is primitive.  For p a
Mersenne exponent (2^p - 1 prime), primitive is the same as irreducible, and a
degree-p polynomial with p prime is irreducible iff x^(2^p) = x (mod mu) and
mu has no root in GF(2) (Rabin's test).  The search draws (m, a) from a seeded
generator, takes mu by Berlekamp-Massey (oracle) on one output bit of 3p
steps from a random state, and keeps the first candidate that passes.

    python tests/golden/make_tgfsr_params.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402


def step(x, w, m, r, a):
    """One step on the window (x_k .. x_{k+n-1}): eq. step with these constants."""
    lower = (1 << r) - 1
    upper = ((1 << w) - 1) ^ lower
    y = (x[0] & upper) | (x[1] & lower)
    return x[1:] + [x[m] ^ (y >> 1) ^ (a if y & 1 else 0)]


def output_bits(x, w, m, r, a, steps, bit=0):
    out = []
    for _ in range(steps):
        x = step(x, w, m, r, a)
        out.append((x[-1] >> bit) & 1)
    return np.array(out, np.uint8)


def full_period(mu, p):
    """Rabin's test for a degree-p polynomial, p prime."""
    if O.poly_deg(mu) != p:
        return False
    x = O.poly([1])
    if not np.array_equal(O.x2pow_chain(mu, p, p)[0], x):
        return False
    v = O.to_int(mu)
    return (v & 1) == 1 and bin(v).count("1") % 2 == 1   # mu(0) = 1 and mu(1) = 1


def search(w, n, r, seed, tries=20000):
    p = n * w - r
    rng = np.random.default_rng(seed)
    for t in range(tries):
        m = int(rng.integers(1, n))
        a = int(rng.integers(0, 1 << w)) | (1 << (w - 1))
        x0 = [int(v) for v in rng.integers(0, 1 << w, size=n)]
        L, mu = O.berlekamp_massey(output_bits(x0, w, m, r, a, 3 * p))
        if L == p and full_period(mu, p):
            return m, a, p, t + 1
    raise RuntimeError(f"no full-period parameters for w={w} n={n} r={r} in {tries} tries")


def main():
    lines = ["# w n m r a p   (twisted GFSR of eq. step, period 2^p - 1; found by make_tgfsr_params.py)"]
    for w, n, r, seed in [(32, 4, 1, 127), (32, 17, 23, 521)]:
        m, a, p, tries = search(w, n, r, seed)
        lines.append(f"{w} {n} {m} {r} 0x{a:08X} {p}")
        print(f"w={w} n={n} r={r}: m={m} a=0x{a:08X} p={p} after {tries} candidates")
    with open(os.path.join(HERE, "tgfsr_params.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
