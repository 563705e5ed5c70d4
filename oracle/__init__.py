"""CPU oracle for the V-family generators (arXiv 2309.16682).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or executes anything here, and
this package never touches the CUDA library.

The arithmetic lives in ``vmt_oracle.c`` (plain scalar C, one function per
paper equation).  This module builds it with gcc, binds it with ctypes and
assembles the V-family stream from it:

* Sec. 3, eq. (subseq)/(combseq): the base stream Z is cut into M sub-sequences
  of length J = ceil(P/M) = 2^(19937 - log2 M) (Table "jvalues"); lane t starts
  at z_{tJ} and the combined sequence S polls the lanes round robin,
  S[kM + t] = z_{tJ + k}.
* Sec. 3, construction of the V generator: lane t's initial state is the base
  state X_0 advanced by tJ steps (plus an optional offset d applied to every
  lane, the ``jump`` argument of ``vmt_init``).
* Sec. 3.1: the advance is the polynomial jump c(F) X_0 with
  c = x^(d + tJ) mod mu, mu the minimal polynomial of F.  The powers
  x^(2^q) mod mu are a chain of squarings; x^e is the product of the chain
  entries at the set bits of e.

For SFMT19937 the interleave unit is the 128-bit element (the paper's w = 128):
S holds uint32 sub-words and element (k, t) occupies S[4(kM + t) + j].

Output conversions (not in the paper; these are readings where it is silent):
``u32`` the words; ``u64`` two consecutive words, the first as the low half
(32-bit variants) or the word itself (MT19937-64); ``f32`` (u >> 8) * 2^-24
(32-bit words) or (u >> 40) * 2^-24 (64-bit words); ``f64``
((a >> 5) * 2^26 + (b >> 6)) * 2^-53 from two consecutive 32-bit words, or
(u >> 11) * 2^-53 from one 64-bit word.

Every function is pinned in tests/test_oracle_*.py.  SFMT19937 seeding is
pinned to numpy's MT19937 legacy seeding over its 624 sub-words; against
upstream SFMT output vectors it is parity unpinned (none available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vmt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MT32, MT64, SFMT = 0, 1, 2
VARIANTS = {"mt32": MT32, "mt64": MT64, "sfmt": SFMT}
N_UNITS = {MT32: 624, MT64: 312, SFMT: 156}       # ring units (words / elements)
WORD_DTYPE = {MT32: np.uint32, MT64: np.uint64, SFMT: np.uint32}
WORDS_PER_UNIT = {MT32: 1, MT64: 1, SFMT: 4}      # native output words per unit
STATE_WORDS = {MT32: 624, MT64: 312, SFMT: 624}   # native words in the buffer
PERIOD_EXP = 19937                                # P = 2^19937 - 1
NW = 314                                          # uint64 words per polynomial

_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile vmt_oracle.c into _build/liboracle.so (plain -O2, no SIMD flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lib_lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.or_seed.argtypes = [ctypes.c_int, P, u64p, ctypes.c_uint64]
            L.or_outputs.argtypes = [ctypes.c_int, P, u64p, P, ctypes.c_int64]
            L.or_raw.argtypes = [ctypes.c_int, P, u64p, P, ctypes.c_int64]
            L.or_jump.argtypes = [ctypes.c_int, P, u64p, P, ctypes.c_int]
            L.or_step_many.argtypes = [ctypes.c_int, P, u64p, ctypes.c_uint64]
            L.or_poly_deg.argtypes = [P, ctypes.c_int]
            L.or_poly_deg.restype = ctypes.c_int
            L.or_poly_mulmod.argtypes = [P, P, P, P, ctypes.c_int]
            L.or_poly_sqrmod.argtypes = [P, P, P, ctypes.c_int]
            L.or_poly_mod.argtypes = [P, ctypes.c_int, P, ctypes.c_int]
            L.or_poly_x2pow_chain.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int]
            L.or_berlekamp_massey.argtypes = [P, ctypes.c_int64, P, ctypes.c_int]
            L.or_berlekamp_massey.restype = ctypes.c_int
            L.or_sfmt_inner.argtypes = [P, ctypes.c_uint64]
            L.or_sfmt_inner.restype = ctypes.c_int
            L.or_mt32_temper.argtypes = [ctypes.c_uint32]
            L.or_mt32_temper.restype = ctypes.c_uint32
            L.or_mt64_temper.argtypes = [ctypes.c_uint64]
            L.or_mt64_temper.restype = ctypes.c_uint64
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# base generators
# ---------------------------------------------------------------------------
class State:
    """Circular buffer of the base generator plus the index k of its oldest word."""

    def __init__(self, variant: int, words: np.ndarray, k: int = 0):
        self.variant = variant
        self.words = np.ascontiguousarray(words, dtype=WORD_DTYPE[variant]).copy()
        assert self.words.size == STATE_WORDS[variant]
        self.k = int(k)

    def copy(self) -> "State":
        return State(self.variant, self.words, self.k)

    def canonical(self) -> np.ndarray:
        """Buffer rotated so that the oldest unit comes first."""
        u = WORDS_PER_UNIT[self.variant]
        n = N_UNITS[self.variant]
        r = self.k % n
        return np.roll(self.words, -r * u)


def seed_state(variant: int, seed: int) -> State:
    st = State(variant, np.zeros(STATE_WORDS[variant], WORD_DTYPE[variant]))
    k = ctypes.c_uint64(0)
    lib().or_seed(variant, _ptr(st.words), ctypes.byref(k), ctypes.c_uint64(seed & (2**64 - 1)))
    st.k = k.value
    return st


def outputs(st: State, units: int) -> np.ndarray:
    """Next `units` outputs of the base generator (advances st).  For SFMT each
    unit is one 128-bit element, returned as 4 uint32 sub-words."""
    v = st.variant
    out = np.zeros(units * WORDS_PER_UNIT[v], WORD_DTYPE[v])
    k = ctypes.c_uint64(st.k)
    lib().or_outputs(v, _ptr(st.words), ctypes.byref(k), _ptr(out), units)
    st.k = k.value
    return out


def raw_words(st: State, units: int) -> np.ndarray:
    v = st.variant
    out = np.zeros(units * WORDS_PER_UNIT[v], WORD_DTYPE[v])
    k = ctypes.c_uint64(st.k)
    lib().or_raw(v, _ptr(st.words), ctypes.byref(k), _ptr(out), units)
    st.k = k.value
    return out


def step_many(st: State, d: int) -> State:
    s = st.copy()
    k = ctypes.c_uint64(s.k)
    lib().or_step_many(s.variant, _ptr(s.words), ctypes.byref(k), ctypes.c_uint64(d))
    s.k = k.value
    return s


def jump(st: State, c: np.ndarray) -> State:
    """Return c(F) st (Horner's rule, Sec. 3.1)."""
    s = st.copy()
    c = np.ascontiguousarray(c, dtype=np.uint64)
    k = ctypes.c_uint64(s.k)
    lib().or_jump(s.variant, _ptr(s.words), ctypes.byref(k), _ptr(c), int(c.size))
    s.k = k.value
    return s


def sfmt_inner(st: State) -> int:
    return lib().or_sfmt_inner(_ptr(st.words), ctypes.c_uint64(st.k))


# ---------------------------------------------------------------------------
# GF(2)[x] polynomials (uint64 words, bit i = coefficient of x^i)
# ---------------------------------------------------------------------------
def poly(bits) -> np.ndarray:
    """Polynomial with the given exponents set."""
    p = np.zeros(NW, np.uint64)
    for e in bits:
        p[e >> 6] ^= np.uint64(1) << np.uint64(e & 63)
    return p


def poly_deg(p: np.ndarray) -> int:
    p = np.ascontiguousarray(p, dtype=np.uint64)
    return lib().or_poly_deg(_ptr(p), int(p.size))


def poly_mulmod(a, b, mu) -> np.ndarray:
    out = np.zeros(NW, np.uint64)
    a = np.ascontiguousarray(a, np.uint64)
    b = np.ascontiguousarray(b, np.uint64)
    mu = np.ascontiguousarray(mu, np.uint64)
    lib().or_poly_mulmod(_ptr(out), _ptr(a), _ptr(b), _ptr(mu), NW)
    return out


def poly_mod(p, mu) -> np.ndarray:
    p = np.ascontiguousarray(p, np.uint64).copy()
    mu = np.ascontiguousarray(mu, np.uint64)
    lib().or_poly_mod(_ptr(p), int(p.size), _ptr(mu), int(mu.size))
    return p[:NW].copy() if p.size >= NW else np.concatenate([p, np.zeros(NW - p.size, np.uint64)])


def berlekamp_massey(bits: np.ndarray) -> tuple[int, np.ndarray]:
    s = np.ascontiguousarray(bits, dtype=np.uint8)
    mu = np.zeros(NW, np.uint64)
    L = lib().or_berlekamp_massey(_ptr(s), int(s.size), _ptr(mu), NW)
    return L, mu


def x2pow_chain(mu: np.ndarray, q_lo: int, q_hi: int) -> np.ndarray:
    out = np.zeros((q_hi - q_lo + 1, NW), np.uint64)
    mu = np.ascontiguousarray(mu, np.uint64)
    lib().or_poly_x2pow_chain(_ptr(out), q_lo, q_hi, _ptr(mu), NW)
    return out


def _gf2_gcd(a: int, b: int) -> int:
    """gcd of two GF(2)[x] polynomials held as Python ints (bit i = x^i)."""
    while b:
        db = b.bit_length()
        while a and a.bit_length() >= db:
            a ^= b << (a.bit_length() - db)
        a, b = b, a
    return a


def _gf2_mul(a: int, b: int) -> int:
    r = 0
    while b:
        low = b & -b
        r ^= a << (low.bit_length() - 1)
        b ^= low
    return r


def _gf2_div(a: int, b: int) -> int:
    q = 0
    db = b.bit_length()
    while a and a.bit_length() >= db:
        s = a.bit_length() - db
        q ^= 1 << s
        a ^= b << s
    assert a == 0
    return q


def to_int(p: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(p, np.uint64).astype("<u8").tobytes(), "little")


def from_int(x: int) -> np.ndarray:
    b = x.to_bytes(NW * 8, "little")
    return np.frombuffer(b, dtype="<u8").astype(np.uint64)


# ---------------------------------------------------------------------------
# minimal polynomial of F and the squaring chain, computed once and cached
# ---------------------------------------------------------------------------
_BM_SEED = 5489
_BM_LEN = 2 * 19968 + 256
_CHAIN_LO = 256          # chain entries 0..255 are stored
_CHAIN_HI_FROM = 19900   # and 19900..19937

_cache: dict[int, dict] = {}
_cache_lock = threading.Lock()
_variant_locks = {v: threading.Lock() for v in (MT32, MT64, SFMT)}


def _bit_sequence(variant: int, bit: int, length: int, seed: int = _BM_SEED) -> np.ndarray:
    """One bit of the raw words of a freshly seeded generator, one per step."""
    st = seed_state(variant, seed)
    w = raw_words(st, length)
    if variant == SFMT:
        w = w.reshape(-1, 4)[:, bit // 32]
        b = bit % 32
    else:
        b = bit
    return ((w >> WORD_DTYPE[variant](b)) & WORD_DTYPE[variant](1)).astype(np.uint8)


def _compute_minpoly(variant: int) -> np.ndarray:
    """mu = lcm of the Berlekamp-Massey polynomials of several output bits.

    For MT19937-32/64 one bit suffices (the polynomial is irreducible of degree
    19937); SFMT19937 has extra small factors, so the lcm over bits 0, 1, ...
    of each sub-word is taken until it stops growing and reaches full degree
    or all 32 candidate bits were used."""
    if variant in (MT32, MT64):
        top = 31 if variant == MT32 else 63
        L, mu = berlekamp_massey(_bit_sequence(variant, top, _BM_LEN))
        return mu
    acc = 1
    for bit in [0, 32, 64, 96, 1, 33, 65, 97, 7, 45, 83, 121, 16, 50, 90, 127]:
        L, mu = berlekamp_massey(_bit_sequence(variant, bit, _BM_LEN))
        m = to_int(mu)
        g = _gf2_gcd(acc, m)
        acc = _gf2_mul(acc, _gf2_div(m, g))
        if acc.bit_length() - 1 >= 32 * 624:
            break
    return from_int(acc)


def _cache_file(variant: int) -> str:
    return os.path.join(_BUILD, f"oracle_poly_v{variant}.npz")


def polys(variant: int) -> dict:
    """{'mu': mu, 'lo': x^(2^q) for q<256, 'hi': x^(2^q) for q in 19900..19937}."""
    with _cache_lock:
        if variant in _cache:
            return _cache[variant]
    with _variant_locks[variant]:
        with _cache_lock:
            if variant in _cache:
                return _cache[variant]
        path = _cache_file(variant)
        src_mtime = os.path.getmtime(_SRC)
        d = None
        if os.path.exists(path) and os.path.getmtime(path) >= src_mtime:
            z = np.load(path)
            d = {"mu": z["mu"], "lo": z["lo"], "hi": z["hi"]}
        if d is None:
            mu = _compute_minpoly(variant)
            chain_lo = x2pow_chain(mu, 0, _CHAIN_LO - 1)
            chain_hi = x2pow_chain(mu, _CHAIN_HI_FROM, PERIOD_EXP)
            d = {"mu": mu, "lo": chain_lo, "hi": chain_hi}
            os.makedirs(_BUILD, exist_ok=True)
            tmp = path + f".tmp{os.getpid()}.npz"
            np.savez(tmp, **d)
            os.replace(tmp, path)
        with _cache_lock:
            _cache[variant] = d
        return d


def prepare_all() -> None:
    """Compute the three variants' tables in parallel (ctypes drops the GIL)."""
    ts = [threading.Thread(target=polys, args=(v,)) for v in (MT32, MT64, SFMT)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()


def minpoly(variant: int) -> np.ndarray:
    return polys(variant)["mu"]


def x2pow(variant: int, q: int) -> np.ndarray:
    d = polys(variant)
    if q < _CHAIN_LO:
        return d["lo"][q]
    if _CHAIN_HI_FROM <= q <= PERIOD_EXP:
        return d["hi"][q - _CHAIN_HI_FROM]
    raise ValueError(f"x^(2^{q}) is not in the cached chain")


def xpow(variant: int, e: int) -> np.ndarray:
    """x^e mod mu: product of the chain entries at the set bits of e."""
    mu = minpoly(variant)
    acc = poly([0])
    q = 0
    while e:
        if e & 1:
            acc = poly_mulmod(acc, x2pow(variant, q), mu)
        e >>= 1
        q += 1
    return acc


def lane_spacing(M: int) -> int:
    """J = ceil(P / M) = 2^(19937 - log2 M) for M a power of two (Table jvalues)."""
    assert M >= 1 and (M & (M - 1)) == 0
    P = 2**PERIOD_EXP - 1
    return -(-P // M)


def jump_by(st: State, e: int) -> State:
    return jump(st, xpow(st.variant, e))


# ---------------------------------------------------------------------------
# V-family stream (Sec. 3)
# ---------------------------------------------------------------------------
def lane_states(variant: int, M: int, seed: int, d: int = 0) -> list[State]:
    """Lane t = X_0 advanced by d + tJ (Sec. 3, V-generator construction)."""
    X0 = seed_state(variant, seed)
    J = lane_spacing(M)
    return [jump_by(X0, d + t * J) if (d + t * J) else X0.copy() for t in range(M)]


def vstream_words(variant: int, M: int, seed: int, count: int, start: int = 0,
                  d: int = 0, lanes: list[State] | None = None) -> np.ndarray:
    """Native words S[start : start + count] of the V-family stream (eq. combseq)."""
    wpu = WORDS_PER_UNIT[variant]
    end = start + count
    rows = -(-end // (wpu * M)) if end else 0
    sts = [s.copy() for s in (lanes if lanes is not None else lane_states(variant, M, seed, d))]
    per_lane = [outputs(s, rows).reshape(rows, wpu) for s in sts]   # [rows, wpu] per lane
    S = np.stack(per_lane, axis=1).reshape(-1)                        # [rows, M, wpu]
    return S[start:end].copy()


def words_per_output(variant: int, dtype: str) -> int:
    if variant == MT64:
        if dtype == "u32":
            raise ValueError("u32 output is not defined for MT19937-64")
        return 1
    return 2 if dtype in ("u64", "f64") else 1


def convert(variant: int, words: np.ndarray, dtype: str) -> np.ndarray:
    """Output conversion of a native word stream (readings in the module doc)."""
    if variant == MT64:
        w = words.astype(np.uint64)
        if dtype == "u64":
            return w.copy()
        if dtype == "f64":
            return (w >> np.uint64(11)).astype(np.float64) * 2.0**-53
        if dtype == "f32":
            return ((w >> np.uint64(40)).astype(np.float64) * 2.0**-24).astype(np.float32)
        raise ValueError(dtype)
    w = words.astype(np.uint32)
    if dtype == "u32":
        return w.copy()
    if dtype == "f32":
        return ((w >> np.uint32(8)).astype(np.float64) * 2.0**-24).astype(np.float32)
    if dtype == "u64":
        a = w[0::2].astype(np.uint64)
        b = w[1::2].astype(np.uint64)
        return a | (b << np.uint64(32))
    if dtype == "f64":
        a = (w[0::2] >> np.uint32(5)).astype(np.float64)
        b = (w[1::2] >> np.uint32(6)).astype(np.float64)
        return (a * 67108864.0 + b) * 2.0**-53
    raise ValueError(dtype)


def vstream(variant: int, M: int, seed: int, count: int, dtype: str, start_word: int = 0,
            d: int = 0, lanes: list[State] | None = None) -> np.ndarray:
    """`count` outputs of type dtype starting at native word index start_word."""
    wpo = words_per_output(variant, dtype)
    w = vstream_words(variant, M, seed, count * wpo, start_word, d, lanes)
    return convert(variant, w, dtype)
