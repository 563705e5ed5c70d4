"""The seeded input recipe (CPU): splitmix64 slices, workload seeds and the
served-mix trace have the properties the benchmark and the tests rely on."""
import math

import numpy as np

from paper_2309_16682_gb300 import inputs as I


def test_splitmix64_slices_agree_with_the_full_sequence():
    full = I.splitmix64(12345, 1000)
    assert np.array_equal(I.splitmix64(12345, 100, first=250), full[250:350])
    assert [int(x) for x in full[:5]] == I.splitmix64_scalar(12345, 5)


def test_workload_seed_modes():
    assert np.all(I.workload_seeds("vmt32_m4_single") == 5489)
    s = I.workload_seeds("vmt64_m8_g32768")
    assert s.size == 32768 and int(s[0]) == 5489 and int(s[-1]) == 5489 + 32767
    s = I.workload_seeds("vmt32_m16_g65536")
    assert s.size == 65536 and np.array_equal(s, I.splitmix64(1, 65536))
    assert np.unique(s).size == s.size


def test_request_trace_matches_its_definition():
    n = 100_000
    tr = I.request_trace(n)
    again = I.request_trace(n)
    assert all(np.array_equal(tr[k], again[k]) for k in tr)                    # seeded
    gaps = np.diff(tr["arrival_s"])
    assert tr["arrival_s"][0] == 0.0 and np.all(gaps >= 0)
    assert abs(gaps.mean() * 2.0e4 - 1.0) < 0.02                              # Poisson at 2e4/s
    assert abs(np.median(gaps) * 2.0e4 - math.log(2)) < 0.03                   # exponential gaps
    assert set(np.unique(tr["variant"])) == {0, 1, 2}
    assert set(np.unique(tr["lanes"])) == {4, 8, 16}
    for k in (0, 1, 2):
        assert abs(np.mean(tr["variant"] == k) - 1 / 3) < 0.01
    assert tr["n"].min() >= 1000 and tr["n"].max() < 10**8
    logs = np.log10(tr["n"])
    assert abs(np.median(logs) - 5.5) < 0.05                                  # log-uniform in [3, 8]
    assert np.unique(tr["seed"]).size > n - 5 and np.unique(tr["jump"]).size > n - 5
