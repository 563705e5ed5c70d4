"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer outputs must match bit for bit; float outputs are exact conversions of
the same bits, so they must match exactly too (tolerance 0).  Small cases are
compared element by element over several blocks with ragged tails; the
full-size workloads are compared on sampled generators (first, last and a
seeded random sample), each checked over its whole output.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_16682_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VNAME = {O.MT32: "mt32", O.MT64: "mt64", O.SFMT: "sfmt"}
VID = {v: k for k, v in VNAME.items()}


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


def _expected(variant, M, seed, segments, d=0, lanes=None):
    """Oracle outputs for consecutive segments [(n, dtype), ...] from word 0."""
    out, w = [], 0
    lanes = lanes if lanes is not None else O.lane_states(variant, M, seed, d)
    total_words = sum(n * O.words_per_output(variant, dt) for n, dt in segments)
    words = O.vstream_words(variant, M, seed, total_words, 0, lanes=lanes)
    for n, dt in segments:
        k = n * O.words_per_output(variant, dt)
        out.append(O.convert(variant, words[w:w + k], dt))
        w += k
    return out


def _assert_same(got, ref, what):
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    bad = np.nonzero(got != ref)[0]
    assert bad.size == 0, f"{what}: {bad.size} mismatches, first at {bad[:5]}: got {got[bad[:3]]} want {ref[bad[:3]]}"


def test_workload_vmt32_m4_single_full(vmt, oracle_polys):
    """The 4-lane single-generator workload, compared word for word (2^20 u32)."""
    g = vmt.VGenerator("mt32", 4, [5489])
    got = _np(g.generate(1 << 20, "u32"))[0]
    assert int(got[9999 * 4]) == 4123659995   # lane 0's 10000th output
    ref = _expected(O.MT32, 4, 5489, [(1 << 20, "u32")])[0]
    _assert_same(got, ref, "vmt32_m4")


def test_vmt64_m8_lane0_10000th(vmt, oracle_polys):
    g = vmt.VGenerator("mt64", 8, [5489])
    got = _np(g.generate(10000 * 8, "u64"))[0]
    assert int(got[9999 * 8]) == 9981545732273789042


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
@pytest.mark.parametrize("M", [1, 2, 4, 8, 16])
def test_ragged_resumed_calls(vmt, oracle_polys, variant, M):
    """Several generators, calls of awkward sizes that resume mid-block."""
    seeds = I.splitmix64(100 + M, 3)
    B = O.N_UNITS[variant] * M * O.WORDS_PER_UNIT[variant]
    native = "u64" if variant == O.MT64 else "u32"
    sizes = [1, max(1, M - 1), B + 1, B - 3, 2 * B + 5, 7]
    segs = [(n, native) for n in sizes]
    g = vmt.VGenerator(VNAME[variant], M, seeds)
    got = [_np(g.generate(n, dt)) for n, dt in segs]
    for gi, s in enumerate(seeds):
        ref = _expected(variant, M, int(s), segs)
        for k in range(len(segs)):
            _assert_same(got[k][gi], ref[k], f"{VNAME[variant]} M={M} gen {gi} call {k}")


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_all_output_types_and_fused_segments(vmt, oracle_polys, variant):
    M = 4
    seeds = I.splitmix64(7, 2)
    dts = ["u64", "f64", "f32"] if variant == O.MT64 else ["u32", "f32", "u64", "f64"]
    segs = [(1000 + 8 * i, dt) for i, dt in enumerate(dts)]
    # plain calls, one type at a time
    g = vmt.VGenerator(VNAME[variant], M, seeds)
    got = [_np(g.generate(n, dt)) for n, dt in segs]
    # the same segments fused into one pass on a fresh generator
    g2 = vmt.VGenerator(VNAME[variant], M, seeds)
    fused = [_np(t) for t in g2.generate_multi(segs)]
    for gi, s in enumerate(seeds):
        ref = _expected(variant, M, int(s), segs)
        for k, (n, dt) in enumerate(segs):
            _assert_same(got[k][gi], ref[k], f"{VNAME[variant]} {dt} gen {gi}")
            _assert_same(fused[k][gi], ref[k], f"{VNAME[variant]} fused {dt} gen {gi}")


@pytest.mark.parametrize("variant", [O.MT32, O.SFMT])
def test_pairs_at_odd_offsets(vmt, oracle_polys, variant):
    """u64/f64 from 32-bit words starting at an odd word (generic path)."""
    M = 2
    g = vmt.VGenerator(VNAME[variant], M, [11])
    a = _np(g.generate(3, "u32"))
    b = _np(g.generate(501, "f64"))
    c = _np(g.generate(77, "u64"))
    ref = _expected(variant, M, 11, [(3, "u32"), (501, "f64"), (77, "u64")])
    _assert_same(a[0], ref[0], "head")
    _assert_same(b[0], ref[1], "f64 odd")
    _assert_same(c[0], ref[2], "u64 odd")


def test_single_lane_pairs(vmt, oracle_polys):
    g = vmt.VGenerator("mt32", 1, [5])
    b = _np(g.generate(999, "f64"))
    ref = _expected(O.MT32, 1, 5, [(999, "f64")])
    _assert_same(b[0], ref[0], "mt32 M=1 f64")


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_init_with_jump_offsets(vmt, oracle_polys, variant):
    M = 4
    seeds = np.array([1, 2, 3], np.uint64)
    jumps = np.array([0, 123456789, 2**64 - 1], np.uint64)
    g = vmt.VGenerator(VNAME[variant], M, seeds, jumps)
    n = 2000
    native = "u64" if variant == O.MT64 else "u32"
    got = _np(g.generate(n, native))
    for gi in range(3):
        ref = _expected(variant, M, int(seeds[gi]), [(n, native)], d=int(jumps[gi]))[0]
        _assert_same(got[gi], ref, f"{VNAME[variant]} d={int(jumps[gi])}")


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_jump_call_and_jump_poly(vmt, oracle_polys, variant):
    """vmt_jump with the library's own x^d polynomial, mid-stream."""
    M = 2
    g = vmt.VGenerator(VNAME[variant], M, [42])
    native = "u64" if variant == O.MT64 else "u32"
    _ = g.generate(5, native)
    d = 987654321
    p = vmt.jump_poly(VNAME[variant], d)
    assert np.array_equal(p, O.xpow(variant, d)[:p.size])
    g.jump(p)
    got = _np(g.generate(3000, native))[0]
    lanes = [O.jump(st, O.xpow(variant, d)) for st in O.lane_states(variant, M, 42)]
    words = O.vstream_words(variant, M, 42, 5 + 3000, 0, lanes=lanes)
    # the jump advances every lane; the stream position inside the block is kept
    _assert_same(got, words[5:], "after vmt_jump")


def test_export_import_resume(vmt, oracle_polys):
    g = vmt.VGenerator("mt32", 8, I.splitmix64(3, 4))
    _ = g.generate(777, "u32")
    blob = g.export_state()
    a = _np(g.generate(20000, "u32"))
    g2 = vmt.VGenerator("mt32", 8, I.splitmix64(99, 4))
    g2.import_state(blob)
    b = _np(g2.generate(20000, "u32"))
    assert np.array_equal(a, b)
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(vmt.VMTError):
        g2.import_state(bytes(bad))


@pytest.mark.parametrize("memory", ["pinned", "pageable"])
def test_generate_host_matches_device(vmt, oracle_polys, memory):
    """Pinned buffers are written directly by the kernels, pageable ones
    through staging; both equal the device path, over several calls."""
    seeds = I.splitmix64(5, 6)
    g1 = vmt.VGenerator("mt32", 16, seeds)
    g2 = vmt.VGenerator("mt32", 16, seeds)
    for n, dt in [(100003, "f32"), (7, "u64"), (70001, "u32")]:
        d = _np(g1.generate(n, dt))
        if memory == "pinned":
            h = g2.generate_host(n, dt).numpy()
        else:
            h = np.empty((6, n), dtype={"f32": np.float32, "u64": np.uint64, "u32": np.uint32}[dt])
            g2.generate_host(n, dt, out=h)
        assert np.array_equal(d, h), (memory, n, dt)


def test_zero_and_empty_calls(vmt, oracle_polys):
    g = vmt.VGenerator("sfmt", 4, [9])
    _ = g.generate(0, "u32")
    got = _np(g.generate(100, "u32"))[0]
    ref = _expected(O.SFMT, 4, 9, [(100, "u32")])[0]
    _assert_same(got, ref, "after empty call")


# ---------------------------------------------------------------------------
# full-size workloads: sampled generators, whole outputs
# ---------------------------------------------------------------------------
def _sample(count, k=6, seed=0):
    rng = np.random.default_rng(seed)
    s = {0, count - 1}
    s.update(int(x) for x in rng.integers(0, count, k))
    return sorted(s)


@pytest.mark.parametrize("name", ["vmt32_m16_g65536", "vmt64_m8_g32768", "vsfmt_m4_g16384"])
def test_full_workloads_sampled(vmt, oracle_polys, name):
    w = I.WORKLOADS[name]
    variant = VID[w["variant"]]
    seeds = I.workload_seeds(name)
    g = vmt.VGenerator(w["variant"], w["lanes"], seeds)
    count = w["generators"]
    segs = [(n // count, dt) for dt, n in w["outputs"]]
    outs = g.generate_multi(segs)
    torch.cuda.synchronize()
    for gi in _sample(count, seed=len(name)):
        ref = _expected(variant, w["lanes"], int(seeds[gi]), segs)
        for k, (n, dt) in enumerate(segs):
            _assert_same(_np(outs[k][gi]), ref[k], f"{name} gen {gi} seg {k}")
    del outs
    torch.cuda.empty_cache()


@pytest.mark.parametrize("name", ["vmt32_m16_g65536", "vmt64_m8_g32768", "vsfmt_m4_g16384"])
def test_full_workloads_wide_sample(vmt, oracle_polys, name):
    """1024 seeded random generators plus the first and the last of each
    full-size workload: the first two blocks of each (every lane's jump-ahead
    and the interleave) equal the oracle.  The lane polynomials x^(tJ) are
    the same for every generator, so the oracle computes them once."""
    w = I.WORKLOADS[name]
    variant, M = VID[w["variant"]], w["lanes"]
    seeds = I.workload_seeds(name)
    count = w["generators"]
    g = vmt.VGenerator(w["variant"], M, seeds)
    native = "u64" if variant == O.MT64 else "u32"
    words = 2 * M * {O.MT32: 624, O.MT64: 312, O.SFMT: 624}[variant]
    out = g.generate(words, native)
    rng = np.random.default_rng(2309 + len(name))
    sample = sorted({0, count - 1} | {int(x) for x in rng.choice(count, 1024, replace=False)})
    signed = out.view(torch.int64 if native == "u64" else torch.int32)   # unsigned CUDA indexing is missing
    got = signed[torch.as_tensor(sample, device=out.device)].cpu().numpy().view(
        np.uint64 if native == "u64" else np.uint32)
    # the plain oracle takes up to ~0.7 s per generator: one spawned process per host core
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor

    from helpers.oracle_pool import first_words
    tasks = [(variant, M, int(seeds[gi]), words) for gi in sample]
    with ProcessPoolExecutor(max_workers=len(os.sched_getaffinity(0)), mp_context=mp.get_context("spawn")) as ex:
        refs = list(ex.map(first_words, tasks, chunksize=4))
    for row, (gi, ref) in enumerate(zip(sample, refs)):
        _assert_same(got[row], ref, f"{name} gen {gi}")


@pytest.mark.parametrize("variant,M,threads", [("mt32", 16, 1024), ("mt32", 8, 512), ("mt64", 8, 512),
                                               ("mt64", 16, 1024)])
def test_every_cta_size_gives_the_same_stream(vmt, variant, M, threads):
    seeds = I.splitmix64(77, 5)
    native = "u64" if variant == "mt64" else "u32"
    segs = [(3001, native), (9000, "f32"), (12345, native)]
    prev = vmt.tune_get_kernel(variant, M)
    try:
        vmt.tune_set(variant, M, 0)
        ref = [_np(t) for t in vmt.VGenerator(variant, M, seeds).generate_multi(segs)]
        vmt.tune_set(variant, M, threads)
        got = [_np(t) for t in vmt.VGenerator(variant, M, seeds).generate_multi(segs)]
    finally:
        vmt.tune_set_kernel(variant, M, prev)
    for k in range(len(segs)):
        assert np.array_equal(got[k], ref[k])
    assert vmt.device_status() == 0


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_ragged_then_lockstep(vmt, oracle_polys, variant):
    """Per-generator lengths in one persistent launch, then a lock-step call
    continues every generator from its own position."""
    M = 4
    seeds = I.splitmix64(300 + variant, 5)
    native = "u64" if variant == O.MT64 else "u32"
    g = vmt.VGenerator(VNAME[variant], M, seeds)
    n1 = [0, 2, 1000, 7778, 20000]
    r = [_np(t) for t in g.generate_ragged(n1, native)]
    n2 = 3002
    tail = _np(g.generate(n2, native))
    for gi, s in enumerate(seeds):
        ref = _expected(variant, M, int(s), [(n1[gi] + n2, native)])[0]
        _assert_same(r[gi], ref[:n1[gi]], f"ragged gen {gi}")
        _assert_same(tail[gi], ref[n1[gi]:], f"lock-step after ragged gen {gi}")


def test_batch_and_graph_match_plain_calls(vmt):
    """A batch over three state objects (three kernels), run plainly and
    through a replayed CUDA graph, equals the same calls made one by one."""
    spec = [("mt32", 16, I.splitmix64(1, 2), 5000, "u32"), ("mt64", 8, I.splitmix64(2, 3), 3000, "f64"),
            ("sfmt", 4, I.splitmix64(3, 2), 7004, "u32")]
    gens = [vmt.VGenerator(v, m, s) for v, m, s, _, _ in spec]
    twins = [vmt.VGenerator(v, m, s) for v, m, s, _, _ in spec]
    outs = [torch.empty((len(s), n), dtype=vmt._torch_dtype(dt), device="cuda") for _, _, s, n, dt in spec]
    b = vmt.Batch()
    for gen, out, (_, _, _, n, dt) in zip(gens, outs, spec):
        b.add(gen, n, dt, out)
    for rnd in range(4):
        b.run(graph=rnd >= 2)
        got = [_np(o) for o in outs]
        for k, (twin, (_, _, _, n, dt)) in enumerate(zip(twins, spec)):
            ref = _np(twin.generate(n, dt))
            assert np.array_equal(got[k], ref), (rnd, k)
    b.close()
    assert vmt.device_status() == 0


@pytest.fixture
def jump_kernel_mode(vmt, request):
    """Force every jump launch onto one kernel: 'split' (one sixteen-warp CTA
    per lane-jump), 'compact' (one four-warp CTA per lane-jump over a small
    ring) or 'warp' (one warp per lane-jump)."""
    value = 1 << 40 if request.param == "split" else 0
    old = {v: vmt.tune_jump(v, value) for v in ("mt32", "mt64", "sfmt")}
    oldc = {v: vmt.tune_jump_compact(v, request.param == "compact") for v in ("mt32", "mt64", "sfmt")}
    yield request.param
    for v, x in old.items():
        vmt.tune_jump(v, x)
        vmt.tune_jump_compact(v, oldc[v])


@pytest.mark.parametrize("jump_kernel_mode", ["split", "compact", "warp"], indirect=True)
@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_both_jump_kernels_match_oracle(vmt, oracle_polys, variant, jump_kernel_mode):
    """Seeding, 64-bit offsets (all eight base-256 digits), lane fan-out and a
    random jump polynomial of degree near the state size, each jump kernel
    against the oracle."""
    M = 8
    seeds = np.array([7, 8, 9, 10, 11], np.uint64)
    jumps = np.array([0, 1, 255, 0x0123456789ABCDEF, 2**64 - 1], np.uint64)
    g = vmt.VGenerator(VNAME[variant], M, seeds, jumps)
    native = "u64" if variant == O.MT64 else "u32"
    wpo = O.words_per_output(variant, native)
    n0 = 700
    got0 = _np(g.generate(n0, native))
    nbits = 19900
    poly = np.random.default_rng(17 + variant).integers(0, 2**63, size=312, dtype=np.uint64)
    poly[nbits // 64] &= np.uint64((1 << (nbits % 64)) - 1)
    poly[nbits // 64 + 1:] = 0
    poly[0] |= np.uint64(1)
    g.jump(poly, nbits=nbits)
    got1 = _np(g.generate(n0, native))
    for gi in range(seeds.size):
        lanes = O.lane_states(variant, M, int(seeds[gi]), int(jumps[gi]))
        ref0 = O.vstream_words(variant, M, 0, n0 * wpo, 0, lanes=lanes)
        _assert_same(got0[gi], O.convert(variant, ref0, native), f"{jump_kernel_mode} init g{gi}")
        # the jump advances every lane's state; the position inside the block stays
        jl = [O.jump(st, poly) for st in lanes]
        ref1 = O.vstream_words(variant, M, 0, 2 * n0 * wpo, 0, lanes=jl)
        _assert_same(got1[gi], O.convert(variant, ref1[n0 * wpo:], native), f"{jump_kernel_mode} jump g{gi}")


def test_two_shards_equal_one_run(vmt):
    """Generators split over two objects (as over two ranks) give the same
    outputs as one object holding all of them."""
    from paper_2309_16682_gb300 import shard
    name, per = "vmt32_m16_g65536", 96
    seeds = shard.rank_seeds(name, 1, 0, 2 * per)
    whole = _np(vmt.VGenerator("mt32", 16, seeds).generate(5000, "u32"))
    parts = [_np(vmt.VGenerator("mt32", 16, shard.rank_seeds(name, 2, r, per)).generate(5000, "u32")) for r in range(2)]
    assert np.array_equal(np.concatenate(parts), whole)


@pytest.mark.parametrize("variant,M,dtype", [(O.MT32, 16, "u32"), (O.MT64, 8, "f64"), (O.SFMT, 4, "u32")])
def test_call_longer_than_one_launch_piece(vmt, oracle_polys, variant, M, dtype):
    """One generator asked for more than 2^31 words in one call (the call is
    cut into launches of at most 2^30 words): words around every cut and at
    the end equal the oracle, whose lanes are jumped forward by whole blocks."""
    wpo = O.words_per_output(variant, dtype)
    n = ((1 << 31) + 4099) // wpo
    g = vmt.VGenerator(VNAME[variant], M, [2024])
    out = g.generate(n, dtype)[0]
    lanes0 = O.lane_states(variant, M, 2024)
    row_words = O.WORDS_PER_UNIT[variant] * M                 # one recurrence step of every lane
    for w_at in [(1 << 30) - 700, (1 << 31) - 700, n * wpo - 1500]:
        row = w_at // row_words                               # steps each lane has taken by then
        lanes = [O.jump_by(st, row) for st in lanes0]
        L = 1500
        ref = O.vstream(variant, M, 0, L // wpo, dtype, start_word=w_at - row * row_words, lanes=lanes)
        got = _np(out[w_at // wpo: w_at // wpo + L // wpo])
        _assert_same(got, ref, f"{VNAME[variant]} word {w_at}")


@pytest.mark.parametrize("variant", [O.MT32, O.MT64, O.SFMT])
def test_every_jump_from_1_to_4096_equals_stepping(vmt, oracle_polys, variant):
    """4096 single-lane generators of one seed, generator d initialised with
    offset d (the device's digit-row jumps): each continues the base stream
    exactly d steps in."""
    native = "u64" if variant == O.MT64 else "u32"
    per_step = 4 if variant == O.SFMT else 1                 # output words per recurrence step
    d = np.arange(1, 4097, dtype=np.uint64)
    g = vmt.VGenerator(VNAME[variant], 1, np.full(4096, 5489, np.uint64), d)
    got = _np(g.generate(8, native))                         # [4096, 8]
    base = O.vstream(variant, 1, 5489, (4096 + 2) * per_step + 8, native)
    idx = (d.astype(np.int64) * per_step)[:, None] + np.arange(8)[None, :]
    assert np.array_equal(got, base[idx])


def test_autotuner_searches_every_configuration_and_keeps_results_exact(vmt):
    old = vmt.tune_get_kernel("mt32", 16)
    cands = vmt.tune_kernels("mt32", 16)
    try:
        best, times = vmt.autotune_grid("mt32", 16, 512, [(3000, "u32"), (3000, "f32")], reps=2)
        assert len(times) == len(cands) and all(t > 0 for t in times)
        assert vmt.tune_get_kernel("mt32", 16) == best and times[best] == min(times)
        t, ms = vmt.autotune("mt32", 16, 512, 0, reps=2, segments=[(3000, "u32"), (3000, "f32")])
        assert t in {c["threads"] for c in cands} and ms > 0
        seeds = I.splitmix64(11, 4)
        a = _np(vmt.VGenerator("mt32", 16, seeds).generate(5000, "u32"))
        vmt.tune_set_kernel("mt32", 16, (vmt.tune_get_kernel("mt32", 16) + 1) % len(cands))
        b = _np(vmt.VGenerator("mt32", 16, seeds).generate(5000, "u32"))
        assert np.array_equal(a, b)
    finally:
        vmt.tune_set_kernel("mt32", 16, old)
