"""Pins of the oracle's jump-ahead machinery and of the V-family interleave (CPU).

* minimal polynomial: for MT19937-32/64 it must be irreducible of degree 19937
  (Rabin's test for a prime degree p: x^(2^p) = x mod phi and no root in GF(2));
  since 2^19937 - 1 is prime it is then primitive.  For SFMT19937 it must carry
  exactly one factor of degree 19937 (gcd with x^(2^19937) - x), which a wrong
  shift direction, sub-word order or constant would destroy.
* mu(F) X = 0 on random states (modulo the r = 31 bits of the oldest MT word that
  the recurrence ignores, Sec. 2.1).
* jumps equal brute-force stepping (oracle stepping and libstdc++ discard),
  compose additively, including chain entries x^(2^q) far beyond brute force.
* M successive J-jumps equal one step for MT (M J = 2^19937 = P + 1).
* SFMT certification: the parity functional vanishes on ker psi(F) and not on
  ker phi(F).
* interleave: lane 0 of S is the base stream; lane t equals the base stream
  advanced by tJ through the chained route.
"""
import numpy as np
import pytest

import oracle as O
from conftest import run_stdmt

MT_VARIANTS = [O.MT32, O.MT64]
ALL_VARIANTS = [O.MT32, O.MT64, O.SFMT]


def _ignored_mask(variant):
    """Bits of the canonical state that never influence an output: the low r=31
    bits of the oldest MT word (Sec. 2.1).  Returns a multiplier mask."""
    st_words = O.STATE_WORDS[variant]
    m = np.full(st_words, np.iinfo(O.WORD_DTYPE[variant]).max, dtype=O.WORD_DTYPE[variant])
    if variant == O.MT32:
        m[0] = 0x80000000
    elif variant == O.MT64:
        m[0] = 0xFFFFFFFF80000000
    return m


def _same_state(a: O.State, b: O.State) -> bool:
    m = _ignored_mask(a.variant)
    return np.array_equal(a.canonical() & m, b.canonical() & m)


def _random_state(variant, rng):
    w = rng.integers(0, np.iinfo(O.WORD_DTYPE[variant]).max, size=O.STATE_WORDS[variant],
                     dtype=O.WORD_DTYPE[variant], endpoint=True)
    return O.State(variant, w, int(rng.integers(0, 1000)))


@pytest.mark.parametrize("variant", MT_VARIANTS)
def test_mt_minpoly_is_primitive_of_degree_19937(oracle_polys, variant):
    mu = O.minpoly(variant)
    assert O.poly_deg(mu) == 19937
    mi = O.to_int(mu)
    assert mi & 1 == 1                      # x does not divide mu  (no root 0)
    assert bin(mi).count("1") % 2 == 1      # mu(1) = 1             (no root 1)
    x = O.poly([1])
    assert np.array_equal(O.x2pow(variant, 19937), x)   # x^(2^p) = x mod mu


def test_sfmt_minpoly_has_one_factor_of_degree_19937(oracle_polys):
    mu = O.minpoly(O.SFMT)
    assert O.poly_deg(mu) == 19968
    mi = O.to_int(mu)
    frob = O.to_int(O.x2pow(O.SFMT, 19937)) ^ 0b10          # x^(2^19937) - x mod mu
    g = O._gf2_gcd(mi, frob)
    # strip the linear factors (x, x+1), whose degree also divides 19937
    for lin in (0b10, 0b11):
        while O._gf2_gcd(g, lin) != 1:
            g = O._gf2_div(g, lin)
    assert g.bit_length() - 1 == 19937


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_minpoly_annihilates_random_states(oracle_polys, variant):
    rng = np.random.default_rng(100 + variant)
    mu = O.minpoly(variant)
    for _ in range(3):
        st = _random_state(variant, rng)
        z = O.jump(st, mu)
        m = _ignored_mask(variant)
        assert not np.any(z.canonical() & m)


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_jump_equals_stepping_small(oracle_polys, variant):
    rng = np.random.default_rng(7 + variant)
    st = O.seed_state(variant, 5489)
    ds = list(range(1, 9)) + [623, 624, 625, 4095, 4096] + [int(x) for x in rng.integers(9, 4097, 6)]
    for d in ds:
        assert _same_state(O.jump_by(st, d), O.step_many(st, d)), d


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_jump_equals_stepping_beyond_degree(oracle_polys, variant):
    """d > deg(mu) exercises the reduction mod mu."""
    rng = np.random.default_rng(70 + variant)
    st = _random_state(variant, rng)
    for d in [20000, 123457, int(rng.integers(2**20, 2**22))]:
        assert _same_state(O.jump_by(st, d), O.step_many(st, d)), d


@pytest.mark.parametrize("bits", [32, 64])
def test_jump_matches_libstdcxx_discard(oracle_polys, stdmt, bits):
    variant = O.MT32 if bits == 32 else O.MT64
    for d in [10_000_000, 2**24 + 12345]:
        ref = run_stdmt(stdmt, bits, 5489, d, 50)
        st = O.jump_by(O.seed_state(variant, 5489), d)
        assert [int(x) for x in O.outputs(st, 50)] == ref


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_chain_squarings_compose_on_states(oracle_polys, variant):
    """Two jumps by 2^(q-1) equal one jump by 2^q, for chain entries far beyond
    any brute-force reach (q = 128 and q = 19934)."""
    rng = np.random.default_rng(31 + variant)
    st = _random_state(variant, rng)
    for q in (128, 19934):
        half = O.x2pow(variant, q - 1)
        lhs = O.jump(O.jump(st, half), half)
        assert _same_state(lhs, O.jump(st, O.x2pow(variant, q)))


@pytest.mark.parametrize("variant", ALL_VARIANTS)
def test_jump_composition(oracle_polys, variant):
    rng = np.random.default_rng(17 + variant)
    st = _random_state(variant, rng)
    a, b = int(rng.integers(0, 2**63)) * 2 + 1, int(rng.integers(0, 2**63))
    lhs = O.jump_by(O.jump_by(st, a), b)
    rhs = O.jump_by(st, a + b)
    assert _same_state(lhs, rhs)


@pytest.mark.parametrize("variant", MT_VARIANTS)
def test_M_lane_jumps_make_one_step(oracle_polys, variant):
    """For MT, M * J = 2^19937 = P + 1, so M jumps by J equal a single step."""
    M = 4
    J = O.lane_spacing(M)
    assert J == 2**19935
    cJ = O.xpow(variant, J)
    st = O.seed_state(variant, 99)
    s = st
    for _ in range(M):
        s = O.jump(s, cJ)
    assert _same_state(s, O.step_many(st, 1))


def test_lane_spacing_table():
    # Table jvalues: J = 2^(19937 - log2 M)
    for M, e in [(2, 19936), (4, 19935), (8, 19934), (16, 19933)]:
        assert O.lane_spacing(M) == 2**e


def test_sfmt_certification_properties(oracle_polys):
    mu = O.to_int(O.minpoly(O.SFMT))
    frob = O.to_int(O.x2pow(O.SFMT, 19937)) ^ 0b10
    phi = O._gf2_gcd(mu, frob)
    for lin in (0b10, 0b11):
        while O._gf2_gcd(phi, lin) != 1:
            phi = O._gf2_div(phi, lin)
    psi = O._gf2_div(mu, phi)
    assert psi.bit_length() - 1 == 31
    rng = np.random.default_rng(5)
    seen_nonzero = False
    for _ in range(12):
        X = _random_state(O.SFMT, rng)
        v2 = O.jump(X, O.from_int(phi))     # in ker psi(F)
        assert O.sfmt_inner(v2) == 0
        v1 = O.jump(X, O.from_int(psi))     # in ker phi(F)
        seen_nonzero |= O.sfmt_inner(v1) == 1
    assert seen_nonzero
    # a certified seed has a non-zero component in ker phi(F)
    st = O.seed_state(O.SFMT, 4321)
    assert np.any(O.jump(st, O.from_int(psi)).words)


@pytest.mark.parametrize("variant,M", [(O.MT32, 4), (O.MT64, 2), (O.SFMT, 2)])
def test_interleave_lanes(oracle_polys, variant, M):
    seed = 5489
    wpu = O.WORDS_PER_UNIT[variant]
    rows = 700
    S = O.vstream_words(variant, M, seed, rows * M * wpu)
    S = S.reshape(rows, M, wpu)
    base = O.outputs(O.seed_state(variant, seed), rows).reshape(rows, wpu)
    assert np.array_equal(S[:, 0, :], base)
    # lane t via t chained jumps by J (the other route than x^(tJ) directly)
    cJ = O.xpow(variant, O.lane_spacing(M))
    st = O.seed_state(variant, seed)
    for t in range(1, M):
        st = O.jump(st, cJ)
        lane = O.outputs(st.copy(), rows).reshape(rows, wpu)
        assert np.array_equal(S[:, t, :], lane)


def test_single_lane_is_base_stream(oracle_polys):
    for v in ALL_VARIANTS:
        S = O.vstream_words(v, 1, 77, 3000)
        base = O.outputs(O.seed_state(v, 77), 3000 // O.WORDS_PER_UNIT[v])
        assert np.array_equal(S, base[:3000])


def test_jump_offset_shifts_every_lane(oracle_polys):
    d = 1000
    S = O.vstream_words(O.MT32, 4, 5, 4 * 50, d=d)
    S0 = O.vstream_words(O.MT32, 4, 5, 4 * (50 + d))
    assert np.array_equal(S, S0[4 * d:])
