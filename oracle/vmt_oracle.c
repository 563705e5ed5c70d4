/*
 * vmt_oracle.c -- CPU oracle for the V-family generators of
 * "VMT19937: A SIMD-Friendly Pseudo Random Number Generator based on
 * Mersenne Twister 19937" (arXiv 2309.16682).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, scalar, obviously-correct
 * statement of what the CUDA library computes.  Only tests/, the smoke check
 * in __graft_entry__ and the CPU-baseline leg of bench.py may load it.  It
 * shares no code, header, table or constant generator with the CUDA library
 * under paper_2309_16682_gb300/, and neither side includes the other.
 *
 * Everything here follows the paper's notation:
 *   - eq. (step)      x_{k+n} = x_{k+m} XOR (x_k & h | x_{k+1} & l) * A
 *   - eq. (matmult)   omega * A = omega >> 1, XOR a when omega is odd
 *   - eq. (tempering) y = x ^ ((x >> alpha) & d); y ^= (y << beta) & b;
 *                     y ^= (y << gamma) & c; z = y ^ (y >> delta)
 *     (the paper's first tempering line writes "x" for x_{k+n})
 *   - eq. (stepmod)   the state is a circular buffer of n words and every
 *                     index is taken modulo n
 *   - eq. (sfmt_step) w_{k+N} = w_k ^ (w_k <<< 8) ^ ((w_{k+m} >> 11) & K)
 *                     ^ (w_{k+N-2} >>> 8) ^ (w_{k+N-1} << 18)
 *   - Sec. 3.1        a jump is applied as c(F) X where c = x^d mod mu and mu
 *                     is the minimal polynomial of the transition F; c(F) X is
 *                     evaluated by Horner's rule: acc <- F(acc) ^ c_i X.
 *
 * Parameters: Sec. 2.2 eq. (params) for MT19937-32, Sec. 2.3 eq. (params64)
 * for MT19937-64, Sec. 2.4 eq. (sfmt_params) for SFMT19937.
 *
 * Readings where the paper is silent:
 *   - seeding: the initialisation recurrences of the C++ standard's
 *     mersenne_twister_engine (multiplier 1812433253 for 32-bit words,
 *     6364136223846793005 for 64-bit words); SFMT uses the 32-bit one on its
 *     624 32-bit sub-words, element k holding sub-words 4k..4k+3;
 *   - SFMT sub-word 0 is the least significant 32 bits of a 128-bit element;
 *   - SFMT period certification with the parity vector
 *     (0x00000001, 0, 0, 0x13c9e684): when the parity of w_0 & p is even the
 *     lowest set bit of p is flipped in w_0;
 *   - the minimal polynomial is found by Berlekamp-Massey on one bit of the
 *     generated words (several bits for SFMT, combined by lcm).
 *
 * Parity status: MT19937-32/64 recurrence, tempering and seeding are pinned by
 * library generators (Python's random, numpy, libstdc++) in the tests; the
 * jump is pinned by brute-force stepping, libstdc++'s discard(d) and the
 * composition of jumps (jump(a) then jump(b) equals jump(a + b)).
 * SFMT19937: the recurrence is pinned algebraically (its minimal polynomial
 * must carry a primitive factor of degree 19937) and the certification by
 * its defining properties; SFMT seeding (the 32-bit initialisation over the
 * 624 sub-words) is pinned by numpy's MT19937 key array after its legacy
 * seeding.  Whether that reading matches upstream SFMT output vectors has no
 * published vector in reach: "parity unpinned" in that sense only.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MT32 0
#define OR_MT64 1
#define OR_SFMT 2

/* ------------------------------------------------------------------ */
/* MT19937-32, Sec. 2.2 eq. (params): (w,n,m,r) = (32,624,397,31)      */
/* ------------------------------------------------------------------ */
#define MT32_N 624
#define MT32_M 397
#define MT32_A 0x9908B0DFu
#define MT32_H 0x80000000u /* h = sum_{i=r}^{w-1} 2^i with r = 31 */
#define MT32_L 0x7FFFFFFFu /* l = sum_{i=0}^{r-1} 2^i             */

/* eq. (matmult) */
static uint32_t mt32_times_A(uint32_t om)
{
    if (om & 1u)
        return (om >> 1) ^ MT32_A;
    return om >> 1;
}

/* eq. (tempering) with (alpha,d)=(11,FFFFFFFF) (beta,b)=(7,9D2C5680)
 * (gamma,c)=(15,EFC60000) delta=18 */
uint32_t or_mt32_temper(uint32_t x)
{
    uint32_t y = x ^ ((x >> 11) & 0xFFFFFFFFu);
    y = y ^ ((y << 7) & 0x9D2C5680u);
    y = y ^ ((y << 15) & 0xEFC60000u);
    return y ^ (y >> 18);
}

/* One application of eq. (step) in the circular-buffer form eq. (stepmod).
 * x[k % n] holds the oldest word x_k; it is replaced by x_{k+n}. */
uint32_t or_mt32_advance(uint32_t *x, uint64_t *k)
{
    uint64_t i = *k;
    uint32_t xk = x[i % MT32_N];
    uint32_t xk1 = x[(i + 1) % MT32_N];
    uint32_t xkm = x[(i + MT32_M) % MT32_N];
    uint32_t omega = (xk & MT32_H) | (xk1 & MT32_L);
    uint32_t xn = xkm ^ mt32_times_A(omega);
    x[i % MT32_N] = xn;
    *k = i + 1;
    return xn;
}

/* Seeding (not in the paper): the C++ standard's mersenne_twister_engine
 * initialisation with f = 1812433253. */
void or_mt32_seed(uint32_t *x, uint64_t *k, uint32_t s)
{
    x[0] = s;
    for (uint32_t i = 1; i < MT32_N; i++)
        x[i] = 1812433253u * (x[i - 1] ^ (x[i - 1] >> 30)) + i;
    *k = 0;
}

/* ------------------------------------------------------------------ */
/* MT19937-64, Sec. 2.3 eq. (params64): (w,n,m,r) = (64,312,156,31)    */
/* ------------------------------------------------------------------ */
#define MT64_N 312
#define MT64_M 156
#define MT64_A 0xB5026F5AA96619E9ull
#define MT64_H 0xFFFFFFFF80000000ull /* 33 upper bits */
#define MT64_L 0x000000007FFFFFFFull /* 31 lower bits */

static uint64_t mt64_times_A(uint64_t om)
{
    if (om & 1u)
        return (om >> 1) ^ MT64_A;
    return om >> 1;
}

/* eq. (tempering) with (29,5555555555555555) (17,71D67FFFEDA60000)
 * (37,FFF7EEE000000000) delta=43 */
uint64_t or_mt64_temper(uint64_t x)
{
    uint64_t y = x ^ ((x >> 29) & 0x5555555555555555ull);
    y = y ^ ((y << 17) & 0x71D67FFFEDA60000ull);
    y = y ^ ((y << 37) & 0xFFF7EEE000000000ull);
    return y ^ (y >> 43);
}

uint64_t or_mt64_advance(uint64_t *x, uint64_t *k)
{
    uint64_t i = *k;
    uint64_t xk = x[i % MT64_N];
    uint64_t xk1 = x[(i + 1) % MT64_N];
    uint64_t xkm = x[(i + MT64_M) % MT64_N];
    uint64_t omega = (xk & MT64_H) | (xk1 & MT64_L);
    uint64_t xn = xkm ^ mt64_times_A(omega);
    x[i % MT64_N] = xn;
    *k = i + 1;
    return xn;
}

void or_mt64_seed(uint64_t *x, uint64_t *k, uint64_t s)
{
    x[0] = s;
    for (uint64_t i = 1; i < MT64_N; i++)
        x[i] = 6364136223846793005ull * (x[i - 1] ^ (x[i - 1] >> 62)) + i;
    *k = 0;
}

/* ------------------------------------------------------------------ */
/* SFMT19937, Sec. 2.4 eq. (sfmt_step), eq. (sfmt_params)             */
/* (w, N, m) = (128, 156, 122); K = (DFFFFFEF, DDFECB7F, BFFAFFFF,     */
/* BFFFFFF6).  Element k occupies sub-words 4k..4k+3, sub-word 0 least */
/* significant.                                                       */
/* ------------------------------------------------------------------ */
#define SFMT_N 156
#define SFMT_M 122
static const uint32_t SFMT_K[4] = {0xDFFFFFEFu, 0xDDFECB7Fu, 0xBFFAFFFFu, 0xBFFFFFF6u};
static const uint32_t SFMT_PARITY[4] = {0x00000001u, 0x00000000u, 0x00000000u, 0x13C9E684u};

/* full 128-bit shifts (the paper's triple-angle operators) */
static void sfmt_shl128(uint32_t out[4], const uint32_t in[4], int s)
{
    uint64_t lo = ((uint64_t)in[1] << 32) | in[0];
    uint64_t hi = ((uint64_t)in[3] << 32) | in[2];
    uint64_t nhi = (hi << s) | (lo >> (64 - s));
    uint64_t nlo = lo << s;
    out[0] = (uint32_t)nlo;
    out[1] = (uint32_t)(nlo >> 32);
    out[2] = (uint32_t)nhi;
    out[3] = (uint32_t)(nhi >> 32);
}

static void sfmt_shr128(uint32_t out[4], const uint32_t in[4], int s)
{
    uint64_t lo = ((uint64_t)in[1] << 32) | in[0];
    uint64_t hi = ((uint64_t)in[3] << 32) | in[2];
    uint64_t nlo = (lo >> s) | (hi << (64 - s));
    uint64_t nhi = hi >> s;
    out[0] = (uint32_t)nlo;
    out[1] = (uint32_t)(nlo >> 32);
    out[2] = (uint32_t)nhi;
    out[3] = (uint32_t)(nhi >> 32);
}

/* One SFMT step on the circular buffer w (SFMT_N elements of 4 sub-words):
 * slot k % N (w_k) is replaced by w_{k+N}; the new element is copied to out. */
void or_sfmt_advance(uint32_t *w, uint64_t *k, uint32_t out[4])
{
    uint64_t i = *k;
    const uint32_t *a = &w[4 * (i % SFMT_N)];                /* w_k       */
    const uint32_t *b = &w[4 * ((i + SFMT_M) % SFMT_N)];     /* w_{k+m}   */
    const uint32_t *c = &w[4 * ((i + SFMT_N - 2) % SFMT_N)]; /* w_{k+N-2} */
    const uint32_t *d = &w[4 * ((i + SFMT_N - 1) % SFMT_N)]; /* w_{k+N-1} */
    uint32_t ashl[4], cshr[4], r[4];
    sfmt_shl128(ashl, a, 8);
    sfmt_shr128(cshr, c, 8);
    for (int j = 0; j < 4; j++)
        r[j] = a[j] ^ ashl[j] ^ ((b[j] >> 11) & SFMT_K[j]) ^ cshr[j] ^ (d[j] << 18);
    for (int j = 0; j < 4; j++) {
        w[4 * (i % SFMT_N) + j] = r[j];
        out[j] = r[j];
    }
    *k = i + 1;
}

/* parity of <p, w_0> over the 128 bits of the oldest element */
int or_sfmt_inner(const uint32_t *w, uint64_t k)
{
    const uint32_t *w0 = &w[4 * (k % SFMT_N)];
    uint32_t acc = 0;
    for (int j = 0; j < 4; j++)
        acc ^= w0[j] & SFMT_PARITY[j];
    int par = 0;
    for (int bit = 0; bit < 32; bit++)
        par ^= (int)((acc >> bit) & 1u);
    return par;
}

/* Period certification: if <p, w_0> is even, flip the lowest set bit of p in w_0. */
void or_sfmt_certify(uint32_t *w, uint64_t k)
{
    if (or_sfmt_inner(w, k) == 1)
        return;
    uint32_t *w0 = &w[4 * (k % SFMT_N)];
    for (int j = 0; j < 4; j++)
        for (int bit = 0; bit < 32; bit++)
            if ((SFMT_PARITY[j] >> bit) & 1u) {
                w0[j] ^= 1u << bit;
                return;
            }
}

void or_sfmt_seed(uint32_t *w, uint64_t *k, uint32_t s)
{
    w[0] = s;
    for (uint32_t i = 1; i < 4 * SFMT_N; i++)
        w[i] = 1812433253u * (w[i - 1] ^ (w[i - 1] >> 30)) + i;
    *k = 0;
    or_sfmt_certify(w, 0);
}

/* ------------------------------------------------------------------ */
/* Generic front end used by the Python wrapper.                      */
/* A state is the circular buffer (624 uint32 for MT32 and SFMT, 312  */
/* uint64 for MT64) plus the index k of the oldest word.              */
/* ------------------------------------------------------------------ */

int or_state_bits(int variant) { return variant == OR_MT64 ? 64 * MT64_N : 32 * MT32_N; }

void or_seed(int variant, void *state, uint64_t *k, uint64_t seed)
{
    if (variant == OR_MT32)
        or_mt32_seed((uint32_t *)state, k, (uint32_t)seed);
    else if (variant == OR_MT64)
        or_mt64_seed((uint64_t *)state, k, seed);
    else
        or_sfmt_seed((uint32_t *)state, k, (uint32_t)seed);
}

/* cnt outputs: z_k = g(x_{k+n}) for MT (tempered), the four sub-words of
 * w_{k+N} for SFMT (cnt counts elements; out receives 4*cnt uint32). */
void or_outputs(int variant, void *state, uint64_t *k, void *out, int64_t cnt)
{
    for (int64_t i = 0; i < cnt; i++) {
        if (variant == OR_MT32)
            ((uint32_t *)out)[i] = or_mt32_temper(or_mt32_advance((uint32_t *)state, k));
        else if (variant == OR_MT64)
            ((uint64_t *)out)[i] = or_mt64_temper(or_mt64_advance((uint64_t *)state, k));
        else
            or_sfmt_advance((uint32_t *)state, k, &((uint32_t *)out)[4 * i]);
    }
}

/* The raw (untempered) new words x_{k+n} / w_{k+N}; same layout as or_outputs. */
void or_raw(int variant, void *state, uint64_t *k, void *out, int64_t cnt)
{
    for (int64_t i = 0; i < cnt; i++) {
        if (variant == OR_MT32)
            ((uint32_t *)out)[i] = or_mt32_advance((uint32_t *)state, k);
        else if (variant == OR_MT64)
            ((uint64_t *)out)[i] = or_mt64_advance((uint64_t *)state, k);
        else
            or_sfmt_advance((uint32_t *)state, k, &((uint32_t *)out)[4 * i]);
    }
}

static void advance_once(int variant, void *state, uint64_t *k)
{
    uint32_t tmp[4];
    if (variant == OR_MT32)
        (void)or_mt32_advance((uint32_t *)state, k);
    else if (variant == OR_MT64)
        (void)or_mt64_advance((uint64_t *)state, k);
    else
        or_sfmt_advance((uint32_t *)state, k, tmp);
}

/* ------------------------------------------------------------------ */
/* GF(2)[x] polynomials: uint64 words, bit i of word i/64 = coeff x^i  */
/* ------------------------------------------------------------------ */
#define PW 640 /* words; holds degree < 40960 (products of degree-<20000 polys) */

int or_poly_deg(const uint64_t *a, int nw)
{
    for (int w = nw - 1; w >= 0; w--)
        if (a[w])
            for (int b = 63; b >= 0; b--)
                if ((a[w] >> b) & 1u)
                    return 64 * w + b;
    return -1;
}

static int getbit(const uint64_t *a, int i) { return (int)((a[i >> 6] >> (i & 63)) & 1u); }

/* a ^= (b << s) for polynomials of nw words (bits shifted past nw*64 are dropped) */
static void xor_shifted(uint64_t *a, const uint64_t *b, int nwb, int s, int nwa)
{
    int ws = s >> 6, bs = s & 63;
    for (int i = 0; i < nwb; i++) {
        if (!b[i])
            continue;
        int t = i + ws;
        if (t < nwa)
            a[t] ^= b[i] << bs;
        if (bs && t + 1 < nwa)
            a[t + 1] ^= b[i] >> (64 - bs);
    }
}

/* r = p mod mu by long division from the top coefficient down.
 * p has nwp words and is overwritten; the remainder is left in p. */
void or_poly_mod(uint64_t *p, int nwp, const uint64_t *mu, int nwmu)
{
    int dm = or_poly_deg(mu, nwmu);
    /* mu shifted by 0..63 bits, so that each subtraction is a plain word XOR */
    int nws = nwmu + 1;
    uint64_t *sh = (uint64_t *)calloc((size_t)64 * nws, sizeof(uint64_t));
    for (int b = 0; b < 64; b++)
        xor_shifted(&sh[b * nws], mu, nwmu, b, nws);
    for (int i = or_poly_deg(p, nwp); i >= dm; i--) {
        if (!getbit(p, i))
            continue;
        int s = i - dm;
        const uint64_t *m = &sh[(s & 63) * nws];
        int ws = s >> 6;
        for (int j = 0; j < nws && ws + j < nwp; j++)
            p[ws + j] ^= m[j];
    }
    free(sh);
}

/* out = a * b mod mu (schoolbook product, then long division) */
void or_poly_mulmod(uint64_t *out, const uint64_t *a, const uint64_t *b, const uint64_t *mu, int nw)
{
    uint64_t *p = (uint64_t *)calloc(2 * (size_t)nw + 2, sizeof(uint64_t));
    int nwp = 2 * nw + 2;
    /* a shifted by 0..63 bits */
    int nws = nw + 1;
    uint64_t *sh = (uint64_t *)calloc((size_t)64 * nws, sizeof(uint64_t));
    for (int s = 0; s < 64; s++)
        xor_shifted(&sh[s * nws], a, nw, s, nws);
    int db = or_poly_deg(b, nw);
    for (int i = 0; i <= db; i++) {
        if (!getbit(b, i))
            continue;
        const uint64_t *m = &sh[(i & 63) * nws];
        int ws = i >> 6;
        for (int j = 0; j < nws; j++)
            p[ws + j] ^= m[j];
    }
    free(sh);
    or_poly_mod(p, nwp, mu, nw);
    memcpy(out, p, (size_t)nw * sizeof(uint64_t));
    free(p);
}

/* out = a^2 mod mu; over GF(2) the square of sum a_i x^i is sum a_i x^{2i} */
void or_poly_sqrmod(uint64_t *out, const uint64_t *a, const uint64_t *mu, int nw)
{
    int nwp = 2 * nw + 2;
    uint64_t *p = (uint64_t *)calloc((size_t)nwp, sizeof(uint64_t));
    int da = or_poly_deg(a, nw);
    for (int i = 0; i <= da; i++)
        if (getbit(a, i))
            p[(2 * i) >> 6] |= 1ull << ((2 * i) & 63);
    or_poly_mod(p, nwp, mu, nw);
    memcpy(out, p, (size_t)nw * sizeof(uint64_t));
    free(p);
}

/* Chain of repeated squarings x^(2^q) mod mu for q = 0..q_hi.  Entries with
 * q in [q_lo, q_hi] are copied to out (nw words each). */
void or_poly_x2pow_chain(uint64_t *out, int q_lo, int q_hi, const uint64_t *mu, int nw)
{
    uint64_t *cur = (uint64_t *)calloc((size_t)nw, sizeof(uint64_t));
    uint64_t *nxt = (uint64_t *)calloc((size_t)nw, sizeof(uint64_t));
    cur[0] = 2; /* x */
    if (or_poly_deg(mu, nw) <= 1) {
        /* degenerate modulus: reduce x first */
        uint64_t *p = (uint64_t *)calloc((size_t)nw, sizeof(uint64_t));
        p[0] = 2;
        or_poly_mod(p, nw, mu, nw);
        memcpy(cur, p, (size_t)nw * sizeof(uint64_t));
        free(p);
    }
    for (int q = 0; q <= q_hi; q++) {
        if (q >= q_lo)
            memcpy(&out[(size_t)(q - q_lo) * nw], cur, (size_t)nw * sizeof(uint64_t));
        if (q == q_hi)
            break;
        or_poly_sqrmod(nxt, cur, mu, nw);
        uint64_t *t = cur;
        cur = nxt;
        nxt = t;
    }
    free(cur);
    free(nxt);
}

/* Berlekamp-Massey over GF(2), one byte per bit.  Returns L, the linear
 * complexity of s[0..n), and writes mu(x) = x^L C(1/x) (so that
 * sum_i mu_i s[k+i] = 0 for all k) into mu_out (nw words). */
int or_berlekamp_massey(const uint8_t *s, int64_t n, uint64_t *mu_out, int nw)
{
    uint8_t *C = (uint8_t *)calloc((size_t)n + 1, 1);
    uint8_t *B = (uint8_t *)calloc((size_t)n + 1, 1);
    uint8_t *T = (uint8_t *)calloc((size_t)n + 1, 1);
    C[0] = 1;
    B[0] = 1;
    int64_t L = 0, m = 1;
    for (int64_t i = 0; i < n; i++) {
        uint8_t d = s[i];
        for (int64_t j = 1; j <= L; j++)
            d ^= (uint8_t)(C[j] & s[i - j]);
        if (d == 0) {
            m++;
        } else if (2 * L <= i) {
            memcpy(T, C, (size_t)n + 1);
            for (int64_t j = 0; j + m <= n; j++)
                C[j + m] ^= B[j];
            L = i + 1 - L;
            memcpy(B, T, (size_t)n + 1);
            m = 1;
        } else {
            for (int64_t j = 0; j + m <= n; j++)
                C[j + m] ^= B[j];
            m++;
        }
    }
    memset(mu_out, 0, (size_t)nw * sizeof(uint64_t));
    for (int64_t j = 0; j <= L; j++)
        if (C[j] && L - j < 64 * (int64_t)nw)
            mu_out[(L - j) >> 6] |= 1ull << ((L - j) & 63);
    free(C);
    free(B);
    free(T);
    return (int)L;
}

/* ------------------------------------------------------------------ */
/* Jump (Sec. 3.1): state <- c(F) state by Horner's rule.             */
/* acc starts at zero; for i = deg c .. 0: acc <- F(acc); if c_i,     */
/* acc ^= X, the two circular buffers aligned by their oldest words.  */
/* The result keeps the circular-buffer index of the input.          */
/* ------------------------------------------------------------------ */
void or_jump(int variant, void *state, uint64_t *k, const uint64_t *c, int nwc)
{
    int n_u32 = (variant == OR_MT64) ? 2 * MT64_N : 4 * SFMT_N; /* 624 uint32 either way */
    int units = (variant == OR_MT32) ? MT32_N : (variant == OR_MT64 ? MT64_N : SFMT_N);
    int upw = n_u32 / units; /* uint32 per ring unit: 1, 2 or 4 */
    uint32_t *X = (uint32_t *)state;
    uint32_t *acc = (uint32_t *)calloc((size_t)n_u32, sizeof(uint32_t));
    uint64_t ka = 0;
    for (int i = or_poly_deg(c, nwc); i >= 0; i--) {
        advance_once(variant, acc, &ka);
        if (getbit(c, i)) {
            for (int j = 0; j < units; j++) {
                int sa = (int)((ka + (uint64_t)j) % (uint64_t)units);
                int sx = (int)((*k + (uint64_t)j) % (uint64_t)units);
                for (int u = 0; u < upw; u++)
                    acc[sa * upw + u] ^= X[sx * upw + u];
            }
        }
    }
    /* write back in the input's ring position */
    for (int j = 0; j < units; j++) {
        int sa = (int)((ka + (uint64_t)j) % (uint64_t)units);
        int sx = (int)((*k + (uint64_t)j) % (uint64_t)units);
        for (int u = 0; u < upw; u++)
            X[sx * upw + u] = acc[sa * upw + u];
    }
    free(acc);
}

/* Plain stepping, for brute-force comparisons: d applications of F. */
void or_step_many(int variant, void *state, uint64_t *k, uint64_t d)
{
    for (uint64_t i = 0; i < d; i++)
        advance_once(variant, state, k);
}
