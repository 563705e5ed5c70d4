"""Every compiled generation-kernel configuration against the oracle (GPU).

The tuning table selects, per (variant, lanes), one of several compiled
kernels (phase, in-place or chain form, lanes per CTA, CTA size, store
width); all must
produce the V-stream exactly.  Each configuration runs the same sequence of
calls on fresh generators -- lock-step calls across blocks and partial blocks,
a fused two-segment call (native words then floats), a tiny call, a ragged
call (unit launch, one length per generator) and a call that resumes from the
resulting unequal positions -- and every output is compared with the oracle's
stream, element by element (tolerance 0: floats are exact conversions).
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_16682_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VNAME = {O.MT32: "mt32", O.MT64: "mt64"}


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


def _plan(variant, M, G):
    """The call sequence: (kind, args) with per-generator output counts."""
    B = O.N_UNITS[variant] * M * O.WORDS_PER_UNIT[variant]
    native = "u64" if variant == O.MT64 else "u32"
    flt = "f64" if variant == O.MT64 else "f32"
    ragged = [B // 2 + 37 * g for g in range(G)]
    return [("gen", [(B + 1, native)]),
            ("multi", [(2 * B + 3, native), (B - 5, flt)]),
            ("gen", [(7, native)]),
            ("ragged", (ragged, native)),
            ("gen", [(3 * B, native)]),
            ("multi", [(B + 8, native), (2 * B, flt)])]


def _oracle_outputs(variant, M, seeds, plan):
    """Per call, per generator: the oracle's outputs (list of arrays)."""
    res = []
    words = []
    for s in seeds:
        total = 0
        for kind, args in plan:
            if kind == "ragged":
                ns, dt = args
                total += max(ns) * O.words_per_output(variant, dt)
            else:
                total += sum(n * O.words_per_output(variant, dt) for n, dt in args)
        words.append(O.vstream_words(variant, M, int(s), total, 0))
    cur = [0] * len(seeds)
    for kind, args in plan:
        per_gen = []
        for g in range(len(seeds)):
            segs = [(args[0][g], args[1])] if kind == "ragged" else args
            outs = []
            for n, dt in segs:
                k = n * O.words_per_output(variant, dt)
                outs.append(O.convert(variant, words[g][cur[g]:cur[g] + k], dt))
                cur[g] += k
            per_gen.append(outs)
        res.append(per_gen)
    return res


def _run(vmt, variant, M, seeds, plan):
    g = vmt.VGenerator(VNAME[variant], M, seeds)
    res = []
    for kind, args in plan:
        if kind == "gen":
            (n, dt), = args
            t = _np(g.generate(n, dt))
            res.append([[t[i]] for i in range(len(seeds))])
        elif kind == "multi":
            ts = [_np(t) for t in g.generate_multi(args)]
            res.append([[t[i] for t in ts] for i in range(len(seeds))])
        else:
            ns, dt = args
            ts = g.generate_ragged(ns, dt)
            res.append([[_np(t)] for t in ts])
    torch.cuda.synchronize()
    return res


CASES = [(O.MT32, 16), (O.MT32, 8), (O.MT32, 4), (O.MT64, 16), (O.MT64, 8), (O.MT64, 4)]


@pytest.mark.parametrize("variant,M", CASES)
def test_every_kernel_configuration_matches_the_oracle(vmt, oracle_polys, variant, M):
    G = 3
    seeds = I.splitmix64(900 + 16 * variant + M, G)
    plan = _plan(variant, M, G)
    ref = _oracle_outputs(variant, M, seeds, plan)
    cands = vmt.tune_kernels(VNAME[variant], M)
    assert len(cands) >= 2
    prev = vmt.tune_get_kernel(VNAME[variant], M)
    try:
        for idx, cfg in enumerate(cands):
            vmt.tune_set_kernel(VNAME[variant], M, idx)
            got = _run(vmt, variant, M, seeds, plan)
            for c, (kind, _) in enumerate(plan):
                for gi in range(G):
                    for k, (a, b) in enumerate(zip(got[c][gi], ref[c][gi])):
                        bad = np.nonzero(np.asarray(a) != np.asarray(b))[0]
                        assert a.shape == b.shape and bad.size == 0, \
                            f"{VNAME[variant]} M={M} config {idx} {cfg} call {c} ({kind}) gen {gi} seg {k}: " \
                            f"{bad.size} mismatches, first at {bad[:4]}"
    finally:
        vmt.tune_set_kernel(VNAME[variant], M, prev)
    assert vmt.device_status() == 0


@pytest.mark.parametrize("variant,M,form", [(O.MT32, 16, "chain"), (O.MT64, 8, "chain"), (O.MT32, 16, "inplace"),
                                            (O.MT64, 8, "inplace"), (O.MT64, 16, "inplace")])
def test_more_generators_than_resident_ctas(vmt, oracle_polys, variant, M, form):
    """1500 generators (for the chain form, half- or quarter-generators): two
    lock-step calls in a row (the second continues the states the first wrote
    back), then a ragged call, a persistent launch whose CTAs take generators
    in turn (in place, every next state is fetched into the copy the previous
    one was just written from); checked on the first, a middle and the last
    generator."""
    name = VNAME[variant]
    cands = vmt.tune_kernels(name, M)
    idx = next(i for i, c in enumerate(cands) if c["form"] == form and (form != "chain" or c["lanes_per_cta"] < M))
    prev = vmt.tune_get_kernel(name, M)
    seeds = I.splitmix64(31 + M, 1500)
    native, flt = ("u64", "f64") if variant == O.MT64 else ("u32", "f32")
    segs = [(20000, native), (5000, flt)]
    ragged = [3000 + 11 * (gi % 97) for gi in range(1500)]   # a persistent unit launch
    try:
        vmt.tune_set_kernel(name, M, idx)
        g = vmt.VGenerator(name, M, seeds)
        a = [_np(t) for t in g.generate_multi(segs)]
        b = [_np(t) for t in g.generate_multi(segs)]
        c = [_np(t) for t in g.generate_ragged(ragged, native)]
    finally:
        vmt.tune_set_kernel(name, M, prev)
    wpo = O.words_per_output(variant, flt)
    per_call = 20000 + 5000 * wpo
    for gi in (0, 777, 1499):
        w = O.vstream_words(variant, M, int(seeds[gi]), 2 * per_call + ragged[gi], 0)
        for k, out in enumerate((a, b)):
            base = k * per_call
            assert np.array_equal(out[0][gi], O.convert(variant, w[base:base + 20000], native)), (form, gi, k)
            assert np.array_equal(out[1][gi], O.convert(variant, w[base + 20000:base + per_call], flt)), (form, gi, k)
        assert np.array_equal(c[gi], O.convert(variant, w[2 * per_call:], native)), (form, gi, "ragged")
