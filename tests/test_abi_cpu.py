"""CPU checks of the C-ABI library (no GPU needed).

* libvmt.so loads and exports every function declared in include/vmt.h.
* The library's host polynomial code (Berlekamp-Massey, products modulo mu, the
  squaring chain) agrees with the oracle's independent implementation.  The
  two share no code; agreement on the same inputs checks both.
* Argument errors are reported with VMT_EINVAL before any device work.
"""
import ctypes
import os
import re
import time

import numpy as np
import pytest

import oracle as O
from conftest import ROOT

vmt = pytest.importorskip("paper_2309_16682_gb300")


@pytest.fixture(scope="module")
def L():
    from paper_2309_16682_gb300 import build
    build.build()
    return vmt.lib()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "vmt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vmt_[a-z0-9_]+)\s*\(", src)))


def test_all_declared_symbols_exported(L):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_invalid_arguments_rejected(L):
    h = ctypes.c_void_p()
    seeds = np.array([1], np.uint64)
    assert L.vmt_init_batch(ctypes.byref(h), 7, 4, 1, seeds.ctypes.data, None, None) == vmt.VMT_EINVAL
    assert L.vmt_init_batch(ctypes.byref(h), 0, 3, 1, seeds.ctypes.data, None, None) == vmt.VMT_EINVAL
    assert L.vmt_init_batch(ctypes.byref(h), 0, 4, 0, seeds.ctypes.data, None, None) == vmt.VMT_EINVAL
    assert b"lanes" in L.vmt_last_error() or b"count" in L.vmt_last_error()
    assert L.vmt_generate(None, 10, 0, None, None) == vmt.VMT_EINVAL
    assert L.vmt_state_import(None, None, 0, None) == vmt.VMT_EINVAL
    assert L.vmt_prepare(3, None) == vmt.VMT_EINVAL
    assert L.vmt_measure_store_bw(1024, 1, None, None) == vmt.VMT_EINVAL
    assert L.vmt_stream_generate(1, 1, 0, 10, vmt.DTYPES["u32"], None, None) == vmt.VMT_EINVAL   # u32 from MT64
    assert L.vmt_stream_generate(0, 1, 0, 10, vmt.DTYPES["u32"], None, None) == vmt.VMT_EINVAL   # null output
    assert L.vmt_tune_jump_set(5, 10) == vmt.VMT_EINVAL
    assert L.vmt_selftest_wait(10, None) == vmt.VMT_EINVAL
    assert L.vmt_server_cancel(None, 1) == vmt.VMT_EINVAL
    assert L.vmt_server_inject(None, vmt.VMT_INJECT_ALLOC, 1) == vmt.VMT_EINVAL
    assert L.vmt_scalar_create(ctypes.byref(h), 0, 4, 1, 0, 0, 10) == vmt.VMT_EINVAL    # buffer too small
    assert L.vmt_scalar_next(None, None) == vmt.VMT_EINVAL
    assert L.vmt_server_next_done(None, 0, None) == vmt.VMT_EINVAL
    assert L.vmt_autotune_multi(0, 16, 10, 0, None, None, 1, None, None, None) == vmt.VMT_EINVAL


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_library_bm_matches_oracle_minpoly(L, oracle_polys, variant):
    bits = O._bit_sequence(variant, 31 if variant == O.MT32 else (63 if variant == O.MT64 else 0), O._BM_LEN)
    d, mu = vmt.poly_minpoly(bits)
    ref = O.minpoly(variant)
    assert d == O.poly_deg(ref)
    n = min(mu.size, ref.size)
    assert np.array_equal(mu[:n], ref[:n]) and not mu[n:].any() and not ref[n:].any()


def test_library_mulmod_matches_oracle(L, oracle_polys):
    rng = np.random.default_rng(4)
    for variant in (O.MT32, O.SFMT):
        mu = O.minpoly(variant)
        nw = O.poly_deg(mu) // 64 + 1
        for _ in range(3):
            a = rng.integers(0, 2**63, size=O.NW, dtype=np.uint64)
            b = rng.integers(0, 2**63, size=O.NW, dtype=np.uint64)
            a[nw - 1:] = 0
            b[nw - 1:] = 0
            ref = O.poly_mulmod(a, b, mu)
            got = vmt.poly_mulmod(a[:nw + 1], b[:nw + 1], mu[:nw + 1])
            assert np.array_equal(got, ref[:nw + 1])


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_library_chain_matches_oracle(L, oracle_polys, variant):
    mu = O.minpoly(variant)
    nw = O.poly_deg(mu) // 64 + 1
    got = vmt.poly_x2pow(mu[:nw], 0, 80)
    for q in (0, 1, 5, 31, 64, 80):
        ref = O.x2pow(variant, q)
        assert np.array_equal(got[q], ref[:nw]) and not ref[nw:].any(), q


@pytest.mark.slow
def test_library_full_chain_matches_oracle(L, oracle_polys):
    mu = O.minpoly(O.MT64)
    t = time.time()
    got = vmt.poly_x2pow(mu[:313], 19933, 19937)
    for i, q in enumerate(range(19933, 19938)):
        assert np.array_equal(got[i], O.x2pow(O.MT64, q)[:313]), q
    assert time.time() - t < 120


def test_tuning_table_round_trips_through_a_file(L, tmp_path):
    import paper_2309_16682_gb300 as vmt
    old = vmt.tune_get("mt32", 16)
    try:
        vmt.tune_set("mt32", 16, 1024)
        f = tmp_path / "tune.txt"
        vmt.tune_save(f)
        vmt.tune_set("mt32", 16, 0)
        assert vmt.tune_get("mt32", 16) != 1024
        vmt.tune_load(f)
        assert vmt.tune_get("mt32", 16) == 1024
        bad = tmp_path / "bad.txt"
        bad.write_text("0 16 777\n0 8 512\n")
        with pytest.raises(vmt.VMTError):
            vmt.tune_load(bad)                   # 777 threads is not compiled...
        assert vmt.tune_get("mt32", 8) == 512    # ...but the valid line applied
    finally:
        vmt.tune_set("mt32", 16, old if old in (512, 1024) else 0)
        vmt.tune_set("mt32", 8, 0)


def test_missing_library_fails_loudly(tmp_path):
    """Without libvmt.so every call raises: there is no CPU fallback."""
    import subprocess
    import sys
    code = (
        "import paper_2309_16682_gb300 as v\n"
        f"v.LIB_PATH = {str(tmp_path / 'absent' / 'libvmt.so')!r}\n"
        "for f in (v.lib, lambda: v.jump_poly('mt32', 5), lambda: v.VGenerator('mt32', 4, [1])):\n"
        "    try:\n"
        "        f()\n"
        "    except RuntimeError as e:\n"
        "        assert 'is missing' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('call succeeded without the library')\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"


def test_kernel_configuration_table_lists_selects_and_round_trips(L, tmp_path):
    import paper_2309_16682_gb300 as vmt
    for variant, lanes in [("mt32", 16), ("mt32", 8), ("mt32", 4), ("mt64", 16), ("mt64", 8), ("mt64", 4)]:
        cands = vmt.tune_kernels(variant, lanes)
        assert len(cands) >= 2 and {"phase", "chain"} <= {c["form"] for c in cands}
        for c in cands:
            assert lanes % c["lanes_per_cta"] == 0 and c["store_bytes"] in (8, 16) and c["threads"] % 32 == 0
            # a lane group's row is whole 16-byte vectors
            assert c["lanes_per_cta"] * (8 if variant == "mt64" else 4) >= 16
    assert vmt.tune_kernels("sfmt", 4) == []
    old = vmt.tune_get_kernel("mt64", 8)
    try:
        n = len(vmt.tune_kernels("mt64", 8))
        vmt.tune_set_kernel("mt64", 8, n - 1)
        assert vmt.tune_get_kernel("mt64", 8) == n - 1
        f = tmp_path / "tune6.txt"
        vmt.tune_save(f)
        assert len(f.read_text().split("\n")[1].split()) == 6
        vmt.tune_set_kernel("mt64", 8, 0)
        vmt.tune_load(f)
        assert vmt.tune_get_kernel("mt64", 8) == n - 1
        with pytest.raises(vmt.VMTError):
            vmt.tune_set_kernel("mt64", 8, n)
        bad = tmp_path / "bad6.txt"
        bad.write_text("1 8 1 3 160 16\n")     # three lanes per CTA: not compiled
        with pytest.raises(vmt.VMTError):
            vmt.tune_load(bad)
    finally:
        vmt.tune_set_kernel("mt64", 8, old)


def test_binding_exposes_its_public_calls():
    """Every Python wrapper of the C ABI is present (CPU; no call is made)."""
    import paper_2309_16682_gb300 as vmt
    for name in ["VGenerator", "ScalarGenerator", "Server", "Batch", "Tgfsr", "tgfsr_jump", "tgfsr_generate",
                 "jump_poly", "stream_generate", "prepare", "measure_store_bw", "device_status", "tune_set",
                 "tune_get", "tune_kernels", "tune_set_kernel", "tune_get_kernel", "tune_jump", "tune_jump_compact",
                 "tune_save", "tune_load", "autotune", "autotune_grid", "poly_minpoly", "poly_mulmod", "poly_x2pow"]:
        assert hasattr(vmt, name), name
    for name in ["submit", "submit_many", "requests", "next_done", "next_done_many", "release", "release_many",
                 "poll", "wait", "copy", "cancel", "stats", "close"]:
        assert hasattr(vmt.Server, name), name
