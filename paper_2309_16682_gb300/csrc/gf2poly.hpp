// gf2poly.hpp -- polynomials over GF(2) for the jump-ahead of Sec. 3.1.
//
// A jump by d steps of an F2-linear generator with transition F is the
// polynomial c(x) = x^d mod mu(x) evaluated at F, where mu is the minimal
// polynomial of F (Sec. 3.1 points to polynomial jump-ahead as the faster
// alternative to the jump matrix F^J).  This header holds the host-side
// arithmetic that builds c(x): Berlekamp-Massey for mu, products and squares
// modulo mu, and the chain x^(2^q) mod mu.  Evaluation of c(F) on states runs
// in CUDA kernels (jump.cu).
//
// Representation: little-endian uint64 words, bit i of word i/64 is the
// coefficient of x^i.
#pragma once
#include <cstdint>
#include <vector>

namespace vmt {
namespace gf2 {

using Poly = std::vector<uint64_t>;

int degree(const Poly& a);
int degree(const uint64_t* a, int nw);

// Linear complexity profile of bits[0..n) (bit i = (bits[i/64] >> (i%64)) & 1).
// Returns mu(x) = x^L C(1/x) where C is the connection polynomial, so that
// sum_i mu_i s[k+i] = 0 for every k.
Poly berlekamp_massey(const uint64_t* bits, int64_t n);

// lcm / gcd / exact division on polynomials of modest degree.
Poly gcd(Poly a, Poly b);
Poly mul_plain(const Poly& a, const Poly& b);
Poly div_exact(Poly a, const Poly& b);

// Arithmetic modulo a fixed polynomial mu.
class Modulus {
public:
    explicit Modulus(const Poly& mu);
    int deg() const { return D_; }
    int words() const { return nw_; }           // words of a reduced element
    const Poly& mu() const { return mu_; }
    Poly reduce(const Poly& p) const;            // p of any degree
    Poly mul(const Poly& a, const Poly& b) const;
    Poly sqr(const Poly& a) const;
    Poly x_pow_2q(int q) const;                  // x^(2^q), q squarings
    Poly x_pow(uint64_t e) const;                // square-and-multiply

private:
    void reduce_in_place(std::vector<uint64_t>& p) const;
    Poly mu_;
    int D_;
    int nw_;
    int bq_;                         // byte index with 8*bq_ >= D_
    int row_bytes_;                  // bytes of a reduction-table row
    std::vector<uint8_t> table_;     // 256 rows: b(x) * x^(8 bq) mod mu
};

}  // namespace gf2
}  // namespace vmt
