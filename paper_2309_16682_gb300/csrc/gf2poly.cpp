// gf2poly.cpp -- host arithmetic in GF(2)[x] for the polynomial jump-ahead
// (Sec. 3.1).  See gf2poly.hpp for the representation.
#include "gf2poly.hpp"

#include <algorithm>
#include <cstring>
#include <stdexcept>

namespace vmt {
namespace gf2 {

static inline int popc64(uint64_t v) { return __builtin_popcountll(v); }
static inline int clz64(uint64_t v) { return __builtin_clzll(v); }

int degree(const uint64_t* a, int nw)
{
    for (int w = nw - 1; w >= 0; --w)
        if (a[w]) return 64 * w + 63 - clz64(a[w]);
    return -1;
}

int degree(const Poly& a) { return degree(a.data(), static_cast<int>(a.size())); }

static inline void trim(Poly& a)
{
    while (!a.empty() && a.back() == 0) a.pop_back();
}

// 64 bits of r starting at bit position pos (r padded by one word).
static inline uint64_t bits_at(const std::vector<uint64_t>& r, int64_t pos)
{
    const int64_t w = pos >> 6;
    const int s = static_cast<int>(pos & 63);
    uint64_t v = r[w] >> s;
    if (s) v |= r[w + 1] << (64 - s);
    return v;
}

// a ^= b << sh, over the first na words of a
static inline void xor_shl(uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int64_t sh)
{
    const int64_t ws = sh >> 6;
    const int bs = static_cast<int>(sh & 63);
    for (int64_t i = 0; i < nb; ++i) {
        const uint64_t v = b[i];
        if (!v) continue;
        const int64_t t = i + ws;
        if (t < na) a[t] ^= v << bs;
        if (bs && t + 1 < na) a[t + 1] ^= v >> (64 - bs);
    }
}

Poly berlekamp_massey(const uint64_t* bits, int64_t n)
{
    // The discrepancy sum_{i=0}^{L} c_i s_{k-i} is the parity of C AND a
    // window of the reversed sequence, evaluated 64 coefficients at a time.
    const int64_t nw = (n + 63) / 64 + 2;
    std::vector<uint64_t> rev(nw + 2, 0);
    for (int64_t i = 0; i < n; ++i)
        if ((bits[i >> 6] >> (i & 63)) & 1ull) {
            const int64_t j = n - 1 - i;
            rev[j >> 6] |= 1ull << (j & 63);
        }
    std::vector<uint64_t> C(nw, 0), B(nw, 0), T;
    C[0] = 1;
    B[0] = 1;
    int64_t L = 0, m = 1, degB = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t off = n - 1 - k;   // rev bit of s_k
        uint64_t acc = 0;
        const int64_t words = L / 64 + 1;
        for (int64_t w = 0; w < words; ++w) acc ^= C[w] & bits_at(rev, off + 64 * w);
        if ((popc64(acc) & 1) == 0) {
            ++m;
            continue;
        }
        if (2 * L <= k) {
            T.assign(C.begin(), C.begin() + std::min<int64_t>(nw, L / 64 + 2));
            const int64_t Told = L;
            xor_shl(C.data(), nw, B.data(), degB / 64 + 1, m);
            L = k + 1 - L;
            std::fill(B.begin(), B.end(), 0);
            std::copy(T.begin(), T.end(), B.begin());
            degB = Told;
            m = 1;
        } else {
            xor_shl(C.data(), nw, B.data(), degB / 64 + 1, m);
            ++m;
        }
    }
    // mu_j = C_{L-j}
    Poly mu((L >> 6) + 1, 0);
    for (int64_t j = 0; j <= L; ++j)
        if ((C[j >> 6] >> (j & 63)) & 1ull) {
            const int64_t e = L - j;
            mu[e >> 6] |= 1ull << (e & 63);
        }
    return mu;
}

static Poly mod_plain(Poly a, const Poly& b)
{
    const int db = degree(b);
    if (db < 0) throw std::invalid_argument("gf2: division by zero");
    for (int i = degree(a); i >= db; --i)
        if ((a[i >> 6] >> (i & 63)) & 1ull) xor_shl(a.data(), static_cast<int64_t>(a.size()), b.data(),
                                                    static_cast<int64_t>(b.size()), i - db);
    trim(a);
    return a;
}

Poly gcd(Poly a, Poly b)
{
    trim(a);
    trim(b);
    while (!b.empty()) {
        Poly r = mod_plain(a, b);
        a = std::move(b);
        b = std::move(r);
    }
    return a;
}

Poly mul_plain(const Poly& a, const Poly& b)
{
    Poly p(a.size() + b.size() + 1, 0);
    const int db = degree(b);
    for (int i = 0; i <= db; ++i)
        if ((b[i >> 6] >> (i & 63)) & 1ull)
            xor_shl(p.data(), static_cast<int64_t>(p.size()), a.data(), static_cast<int64_t>(a.size()), i);
    trim(p);
    return p;
}

Poly div_exact(Poly a, const Poly& b)
{
    const int db = degree(b);
    const int da = degree(a);
    if (db < 0) throw std::invalid_argument("gf2: division by zero");
    Poly q(da >= db ? (da - db) / 64 + 1 : 1, 0);
    for (int i = da; i >= db; --i)
        if ((a[i >> 6] >> (i & 63)) & 1ull) {
            q[(i - db) >> 6] |= 1ull << ((i - db) & 63);
            xor_shl(a.data(), static_cast<int64_t>(a.size()), b.data(), static_cast<int64_t>(b.size()), i - db);
        }
    if (degree(a) >= 0) throw std::runtime_error("gf2: inexact division");
    trim(q);
    return q;
}

// ---------------------------------------------------------------------------
// Modulus
// ---------------------------------------------------------------------------
Modulus::Modulus(const Poly& mu) : mu_(mu)
{
    trim(mu_);
    D_ = degree(mu_);
    if (D_ < 1) throw std::invalid_argument("gf2: modulus of degree < 1");
    nw_ = D_ / 64 + 1;
    mu_.resize(nw_ + 1, 0);
    bq_ = (D_ + 7) / 8;
    row_bytes_ = ((bq_ + 7) / 8) * 8;
    table_.assign(static_cast<size_t>(256) * row_bytes_, 0);
    // rows for single bits: x^(8 bq + u) mod mu, u = 0..7, by plain long division
    std::vector<Poly> single(8);
    for (int u = 0; u < 8; ++u) {
        Poly p(static_cast<size_t>((8 * bq_ + u) / 64 + 2), 0);
        const int e = 8 * bq_ + u;
        p[e >> 6] |= 1ull << (e & 63);
        single[u] = mod_plain(p, mu_);
        single[u].resize(static_cast<size_t>(row_bytes_ / 8), 0);
    }
    for (int b = 1; b < 256; ++b) {
        uint64_t* row = reinterpret_cast<uint64_t*>(&table_[static_cast<size_t>(b) * row_bytes_]);
        for (int u = 0; u < 8; ++u)
            if ((b >> u) & 1)
                for (int w = 0; w < row_bytes_ / 8; ++w) row[w] ^= single[u][w];
    }
}

void Modulus::reduce_in_place(std::vector<uint64_t>& p) const
{
    // room for unaligned 8-byte XORs past the top of any row
    const size_t need = static_cast<size_t>(std::max<int>(nw_ + 2, static_cast<int>(p.size()) + 2));
    p.resize(need, 0);
    uint8_t* bytes = reinterpret_cast<uint8_t*>(p.data());
    const int top = degree(p);
    if (top >= D_) {
        for (int bi = top >> 3; bi >= bq_; --bi) {
            const uint8_t b = bytes[bi];
            if (!b) continue;
            bytes[bi] = 0;
            const uint8_t* row = &table_[static_cast<size_t>(b) * row_bytes_];
            uint8_t* dst = bytes + (bi - bq_);
            for (int o = 0; o < row_bytes_; o += 8) {
                uint64_t x, y;
                std::memcpy(&x, dst + o, 8);
                std::memcpy(&y, row + o, 8);
                x ^= y;
                std::memcpy(dst + o, &x, 8);
            }
        }
        // bits D .. 8 bq - 1 (when D is not a multiple of 8)
        for (int i = 8 * bq_ - 1; i >= D_; --i)
            if ((p[i >> 6] >> (i & 63)) & 1ull)
                xor_shl(p.data(), static_cast<int64_t>(p.size()), mu_.data(), static_cast<int64_t>(mu_.size()),
                        i - D_);
    }
    p.resize(static_cast<size_t>(nw_));
}

Poly Modulus::reduce(const Poly& a) const
{
    Poly p = a;
    reduce_in_place(p);
    return p;
}

Poly Modulus::mul(const Poly& a_in, const Poly& b_in) const
{
    Poly a = reduce(a_in), b = reduce(b_in);
    const int na = nw_ + 1;  // multiples of a by a 4-bit u have degree < D + 3
    std::vector<uint64_t> T(static_cast<size_t>(16) * na, 0);
    for (int u = 1; u < 16; ++u)
        for (int s = 0; s < 4; ++s)
            if ((u >> s) & 1) xor_shl(&T[static_cast<size_t>(u) * na], na, a.data(), nw_, s);
    const int np = 2 * nw_ + 2;
    std::vector<uint64_t> P(static_cast<size_t>(np), 0);
    // left-to-right comb over the 16 nibbles of every word of b
    for (int k = 15; k >= 0; --k) {
        for (int w = 0; w < nw_; ++w) {
            const int nib = static_cast<int>((b[w] >> (4 * k)) & 15u);
            if (!nib) continue;
            const uint64_t* t = &T[static_cast<size_t>(nib) * na];
            uint64_t* dst = &P[w];
            for (int j = 0; j < na; ++j) dst[j] ^= t[j];
        }
        if (k) {
            for (int j = np - 1; j > 0; --j) P[j] = (P[j] << 4) | (P[j - 1] >> 60);
            P[0] <<= 4;
        }
    }
    reduce_in_place(P);
    return P;
}

static const uint16_t* spread_table()
{
    static uint16_t t[256];
    static bool init = false;
    if (!init) {
        for (int b = 0; b < 256; ++b) {
            uint16_t v = 0;
            for (int i = 0; i < 8; ++i)
                if ((b >> i) & 1) v |= static_cast<uint16_t>(1u << (2 * i));
            t[b] = v;
        }
        init = true;
    }
    return t;
}

Poly Modulus::sqr(const Poly& a_in) const
{
    // over GF(2), (sum a_i x^i)^2 = sum a_i x^(2i)
    Poly a = reduce(a_in);
    const uint16_t* sp = spread_table();
    std::vector<uint64_t> P(static_cast<size_t>(2 * nw_ + 2), 0);
    for (int w = 0; w < nw_; ++w) {
        const uint64_t v = a[w];
        uint64_t lo = 0, hi = 0;
        for (int by = 0; by < 4; ++by) lo |= static_cast<uint64_t>(sp[(v >> (8 * by)) & 255]) << (16 * by);
        for (int by = 0; by < 4; ++by) hi |= static_cast<uint64_t>(sp[(v >> (32 + 8 * by)) & 255]) << (16 * by);
        P[2 * w] = lo;
        P[2 * w + 1] = hi;
    }
    reduce_in_place(P);
    return P;
}

Poly Modulus::x_pow_2q(int q) const
{
    Poly x(2, 0);
    x[0] = 2;
    Poly r = reduce(x);
    for (int i = 0; i < q; ++i) r = sqr(r);
    return r;
}

Poly Modulus::x_pow(uint64_t e) const
{
    Poly one(1, 1);
    Poly r = reduce(one);
    Poly x(2, 0);
    x[0] = 2;
    Poly base = reduce(x);
    while (e) {
        if (e & 1) r = mul(r, base);
        e >>= 1;
        if (e) base = sqr(base);
    }
    return r;
}

}  // namespace gf2
}  // namespace vmt
