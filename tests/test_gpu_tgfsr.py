"""The jump kernels of vmt_jump on twisted GFSRs small enough for the matrix
route of Sec. 3.1, and the V-family construction on one of them (GPU).

Sec. 3.1 gives two routes to a jumped state: B = F^J applied to X, and
c(F) X with c = x^J mod the minimal polynomial.  For MT19937 only the second
is feasible.  Here the window-correlation kernels that vmt_jump runs (the
warp form and the CTA form, the same templates with the sequence extended by
a run-time recurrence) jump states of

  * the 80-bit analogue of the CPU matrix cross-check (w = 16, n = 5, m = 2,
    r = 7, a = 0xB4F1), c from the oracle's polynomial routines;
  * the two full-period generators of tests/golden/tgfsr_params.txt (p = 127
    and p = 521), c from the library's own host helpers (Berlekamp-Massey on
    output bits, then x^J by the squaring chain);

and every result must equal F^J X from the matrix power, which shares nothing
with either polynomial code.  On the 521-bit generator a 4-lane V-generator
is built on the GPU (lane t = F^(tJ) X, J = 2^(p-2)), its interleaved
tempered stream compared with plain stepping, and M successive J-jumps
checked to equal one step (M J = 2^p = 1 step modulo the period).
"""
import numpy as np
import pytest

import oracle as O
import test_oracle_matrix_jump as A
import test_tgfsr_cpu as T

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MT_TEMPER = dict(u=11, d=0xFFFFFFFF, s=7, b=0x9D2C5680, t=15, c=0xEFC60000, l=18)


@pytest.fixture(scope="module")
def vmt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_16682_gb300 as m
    from paper_2309_16682_gb300 import build
    build.build()
    m.lib()
    return m


def _params(vmt, g, temper=False):
    p = vmt.Tgfsr()
    p.w, p.n, p.m, p.r, p.a = g["w"], g["n"], g["m"], g["r"], g["a"]
    p.temper = 1 if temper else 0
    if temper:
        for k, v in MT_TEMPER.items():
            setattr(p, k, v)
    return p


def _words(c: int) -> np.ndarray:
    nw = max(1, (c.bit_length() + 63) // 64)
    return np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(nw)], dtype=np.uint64)


def _gpu_states(states):
    a = np.array(states, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()


def _host_states(t):
    return t.cpu().numpy().view(np.uint32).tolist()


ANALOGUE = dict(w=A.W, n=A.N, m=A.MM, r=A.R, a=A.A)


@pytest.mark.parametrize("kernel", ["warp", "cta"])
def test_jump_kernels_equal_the_matrix_power_on_the_80_bit_analogue(vmt, kernel):
    rng = np.random.default_rng(80)
    xs = [A.step([int(v) for v in rng.integers(0, 1 << A.W, size=A.N)]) for _ in range(12)]
    mu = 1
    for x in xs:   # a polynomial that annihilates every state's orbit
        m = A.minimal_polynomial(x)
        mu = O._gf2_div(O._gf2_mul(mu, m), O._gf2_gcd(mu, m))
    F = A.transition_matrix()
    prm = _params(vmt, ANALOGUE)
    for J in [1, 2, 79, 80, 81, 4097, 2**40 + 12345, 2**63 - 1, 3**50, 2**79]:
        c = A.xpow_mod(J, mu)
        st = _gpu_states(xs)
        vmt.tgfsr_jump(prm, st, _words(c), kernel=kernel)
        got = _host_states(st)
        BJ = A.matpow2(F, J)
        for x, y in zip(xs, got):
            assert y == A.from_bits(BJ @ A.to_bits(x) % 2), (J, kernel)


def _library_xpow(vmt, J, mu):
    chain = vmt.poly_x2pow(mu, 0, J.bit_length())
    acc = np.zeros(mu.size, np.uint64)
    acc[0] = 1
    for q in range(J.bit_length()):
        if (J >> q) & 1:
            acc = vmt.poly_mulmod(acc, chain[q], mu)
    return acc


def _library_minpoly(vmt, g, x):
    bits, y = [], x
    for _ in range(3 * g["p"]):
        y = T.step(y, g)
        bits.append(y[-1] & 1)
    d, mu = vmt.poly_minpoly(np.array(bits, np.uint8))
    assert d == g["p"]
    return mu[:d // 64 + 1].copy()


@pytest.mark.parametrize("kernel", ["warp", "cta"])
@pytest.mark.parametrize("g", T.load_params(), ids=lambda g: f"p{g['p']}")
def test_jump_kernels_equal_the_matrix_power_on_full_period_generators(vmt, g, kernel):
    xs = [T.image_state(g, 1000 + i) for i in range(24)]
    mu = _library_minpoly(vmt, g, xs[0])
    F = T.transition(g)
    prm = _params(vmt, g)
    for J in [1, g["p"], 2**64 + 3, 2**200 + 7]:
        st = _gpu_states(xs)
        vmt.tgfsr_jump(prm, st, _library_xpow(vmt, J, mu), kernel=kernel)
        got = _host_states(st)
        BJ = T.mat_pow2(F, J)
        for x, y in zip(xs, got):
            assert y == T.from_bits(BJ @ T.to_bits(x, g), g), (g["p"], J, kernel)


def _temper(y):
    k = MT_TEMPER
    y ^= (y >> k["u"]) & k["d"]
    y ^= (y << k["s"]) & k["b"] & 0xFFFFFFFF
    y ^= (y << k["t"]) & k["c"] & 0xFFFFFFFF
    return (y ^ (y >> k["l"])) & 0xFFFFFFFF


def _stream(g, x, n):
    out = []
    for _ in range(n):
        x = T.step(x, g)
        out.append(_temper(x[-1]))
    return out


def test_v_generator_on_the_521_bit_generator(vmt):
    g = [p for p in T.load_params() if p["p"] == 521][0]
    M, G, K = 4, 6, 3000
    J = 2**(g["p"] - 2)                    # ceil((2^p - 1) / M)
    base = [T.image_state(g, 5000 + i) for i in range(G)]
    mu = _library_minpoly(vmt, g, base[0])
    prm = _params(vmt, g, temper=True)
    states = _gpu_states([x for x in base for _ in range(M)])        # [G * M, n], lane-minor
    for t in range(1, M):
        lane = states[t::M].clone()
        vmt.tgfsr_jump(prm, lane, _library_xpow(vmt, t * J, mu), kernel="cta")
        states[t::M] = lane
    out1 = vmt.tgfsr_generate(prm, states, M, K).cpu().numpy().view(np.uint32)
    out2 = vmt.tgfsr_generate(prm, states, M, 100).cpu().numpy().view(np.uint32)   # the streams continue
    B1 = T.mat_pow2(T.transition(g), J)
    for gi, x in enumerate(base):
        ref0 = _stream(g, x, K + 100)
        assert out1[gi, 0::M].tolist() == ref0[:K] and out2[gi, 0::M].tolist() == ref0[K:]
        x1 = T.from_bits(B1 @ T.to_bits(x, g), g)   # lane 1 = F^J X by the matrix route
        ref1 = _stream(g, x1, K)
        assert out1[gi, 1::M].tolist() == ref1
    # M jumps by J make one step: M J = 2^p, and 2^p = 1 modulo the period
    st = _gpu_states(base)
    cJ = _library_xpow(vmt, J, mu)
    for _ in range(M):
        vmt.tgfsr_jump(prm, st, cJ, kernel="warp")
    assert _host_states(st) == [T.step(x, g) for x in base]


def test_bad_parameters_are_rejected(vmt):
    g = dict(ANALOGUE)
    st = _gpu_states([[0] * 5])
    for bad in [dict(n=6), dict(m=5), dict(r=0), dict(w=33), dict(a=1 << 16)]:
        prm = _params(vmt, dict(g, **bad))
        with pytest.raises(vmt.VMTError):
            vmt.tgfsr_jump(prm, st, np.array([1], np.uint64))
