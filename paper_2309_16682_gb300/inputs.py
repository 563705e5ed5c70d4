"""Seeded synthetic inputs shared by the tests, the oracle side and the benchmark.

This module holds no arithmetic of the generators themselves; it only produces
the *inputs* of the workloads: per-generator seeds, jump offsets and request
traces.  Seeds come from splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the 64-bit finaliser constants
are the published ones):

    state += 0x9E3779B97F4A7C15
    z = (state ^ (state >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    output z ^ (z >> 31)

Generator g of a batch seeded with s receives the g-th output (0-based) of the
splitmix64 sequence that starts from state s.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1


def splitmix64_scalar(state: int, count: int) -> list[int]:
    """Reference form on Python integers."""
    out = []
    s = state & MASK64
    for _ in range(count):
        s = (s + GOLDEN) & MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        out.append(z ^ (z >> 31))
    return out


def splitmix64(state: int, count: int, first: int = 0) -> np.ndarray:
    """Vectorised form: the i-th output only depends on state + (i+1)*GOLDEN,
    so outputs [first, first + count) come without the ones before them."""
    with np.errstate(over="ignore"):
        i = np.arange(first + 1, first + count + 1, dtype=np.uint64)
        s = np.uint64(state & MASK64) + i * np.uint64(GOLDEN)
        z = (s ^ (s >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform01(u64: np.ndarray) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of 64-bit draws."""
    return (u64 >> np.uint64(11)).astype(np.float64) * 2.0**-53


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
WORKLOADS = {
    # name: (variant, lanes, generators, seeds, words per generator per call)
    "vmt32_m4_single": dict(variant="mt32", lanes=4, generators=1, seed_mode="fixed", seed=5489,
                            outputs=[("u32", 1 << 20)]),
    "vmt32_m16_g65536": dict(variant="mt32", lanes=16, generators=65536, seed_mode="splitmix", seed=1,
                             outputs=[("u32", 1 << 30), ("f32", 1 << 30)]),
    "vmt64_m8_g32768": dict(variant="mt64", lanes=8, generators=32768, seed_mode="consecutive", seed=5489,
                            outputs=[("u64", 1 << 29), ("f64", 1 << 29)]),
    "vsfmt_m4_g16384": dict(variant="sfmt", lanes=4, generators=16384, seed_mode="splitmix", seed=1,
                            outputs=[("u32", 1 << 30)]),
}


def workload_seeds(name: str, first: int = 0, count: int | None = None) -> np.ndarray:
    """Seeds of generators [first, first + count) of the workload's global
    generator sequence (count defaults to the workload's generator count).
    With several GPUs each rank takes its own slice of the same sequence."""
    w = WORKLOADS[name]
    n = w["generators"] if count is None else count
    if w["seed_mode"] == "fixed":
        return np.full(n, w["seed"], dtype=np.uint64)
    if w["seed_mode"] == "consecutive":
        # generator g is seeded with seed + g, so generator 0 keeps the named seed
        return np.uint64(w["seed"]) + np.arange(first, first + n, dtype=np.uint64)
    return splitmix64(w["seed"], n, first)


def request_trace(count: int, rate_per_s: float = 2.0e4, seed: int = 2,
                  lanes_choices=(4, 8, 16), n_lo: float = 1e3, n_hi: float = 1e8):
    """Served-mix workload: Poisson arrivals, variant uniform over the three base
    generators, lane width uniform over lanes_choices, output length log-uniform
    in [n_lo, n_hi] native words, per-request seed and 64-bit jump offset.

    All draws come from one splitmix64 stream starting at `seed`; six draws per
    request in a fixed order (arrival gap, variant, lanes, length, seed, jump)."""
    r = splitmix64(seed, 6 * count).reshape(count, 6)
    u_gap = uniform01(r[:, 0])
    gaps = -np.log1p(-u_gap) / rate_per_s
    arrival = np.cumsum(gaps) - gaps[0]
    variant = (r[:, 1] % np.uint64(3)).astype(np.int64)
    lanes = np.asarray(lanes_choices, dtype=np.int64)[(r[:, 2] % np.uint64(len(lanes_choices))).astype(np.int64)]
    u_len = uniform01(r[:, 3])
    n = np.floor(np.exp(math.log(n_lo) + u_len * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    seeds = r[:, 4].copy()
    jumps = r[:, 5].copy()
    return dict(arrival_s=arrival, variant=variant, lanes=lanes, n=n, seed=seeds, jump=jumps)
