// vmt_device.cuh -- device-side building blocks shared by the V-family kernels.
//
// Generators (arXiv 2309.16682):
//   MT19937-32  Sec. 2.2 eq. (params):   (w,n,m,r) = (32,624,397,31), a = 9908B0DF
//   MT19937-64  Sec. 2.3 eq. (params64): (64,312,156,31), a = B5026F5AA96619E9
//   SFMT19937   Sec. 2.4 eq. (sfmt_params): (128,156,122), K = (DFFFFFEF, DDFECB7F,
//               BFFAFFFF, BFFFFFF6)
// Recurrence eq. (step) with the multiplication by A of eq. (matmult), the
// tempering eq. (tempering) and the SFMT recurrence eq. (sfmt_step).
//
// Output conversions are not in the paper; their definitions:
//   f32 from a 32-bit word z:  (z >> 8) * 2^-24           (exact)
//   f32 from a 64-bit word z:  (z >> 40) * 2^-24          (exact)
//   f64 from a 64-bit word z:  (z >> 11) * 2^-53          (exact)
//   f64 from two 32-bit words (a, b):  ((a >> 5) 2^26 + (b >> 6)) 2^-53
//   u64 from two 32-bit words (a, b):  a | b << 32
// The f64 value is assembled from integer fields (no FP64 instruction): the
// 53-bit integer v is normalised with a leading-zero count and its exponent
// written directly, which is exact because v < 2^53.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include "gen_args.hpp"

namespace vmt {
namespace dev {

// ----------------------------------------------------------------------------
// generator constants
// ----------------------------------------------------------------------------
// Pipe balance.  The twist and the tempering are logic operations and
// constant shifts, which share the ALU pipe; on MT19937-64 generation that
// pipe is the bound, while the multiply-add pipe has room.  A left shift by s
// is a multiplication by 2^s, but the compiler turns a multiplication by a
// known power of two back into a shift, so the tempering takes its
// multipliers from ShiftK, which every launch passes as a kernel parameter
// (an operand the compiler cannot see through).  The multiplication by the
// twist constant a (y odd ? a : 0 = (y & 1) * a) is not a power of two and
// stays on the multiply-add pipe by itself.  Right shifts stay on the ALU
// pipe: a multiply-high runs at half the multiply-add rate.

struct MT32 {
    using W = uint32_t;
    static constexpr int N = 624, MM = 397;
    // eq. (step) with y * A of eq. (matmult): y >> 1, XOR a when y is odd;
    // y's lowest bit is the lowest bit of x_{k+1}
    static __device__ __forceinline__ W twist(W xk, W xk1, W xkm)
    {
        const W y = (xk & 0x80000000u) | (xk1 & 0x7FFFFFFFu);
        return xkm ^ (y >> 1) ^ ((xk1 & 1u) * 0x9908B0DFu);
    }
    // eq. (tempering) with (u, s, b, t, c, l) = (11, 7, 9D2C5680, 15, EFC60000, 18)
    static __device__ __forceinline__ W temper(W y)
    {
        y ^= y >> 11;
        y ^= (y << 7) & 0x9D2C5680u;
        y ^= (y << 15) & 0xEFC60000u;
        return y ^ (y >> 18);
    }
    static __device__ __forceinline__ W temper(W y, const ShiftK& k)
    {
        y ^= y >> 11;
        y ^= (y * k.p7) & 0x9D2C5680u;
        y ^= (y * k.p15) & 0xEFC60000u;
        return y ^ (y >> 18);
    }
    static __device__ __forceinline__ W twist(W xk, W xk1, W xkm, const ShiftK&) { return twist(xk, xk1, xkm); }
};

// MT19937-64 on 32-bit halves (lo, hi): every 64-bit shift by a constant is
// one funnel shift plus one 32-bit shift, every mask one operation per half.
__device__ __forceinline__ uint32_t lo32(unsigned long long x) { return static_cast<uint32_t>(x); }
__device__ __forceinline__ uint32_t hi32(unsigned long long x) { return static_cast<uint32_t>(x >> 32); }
__device__ __forceinline__ unsigned long long pack64(uint32_t lo, uint32_t hi)
{
    return (static_cast<unsigned long long>(hi) << 32) | lo;
}

struct MT64 {
    using W = unsigned long long;
    static constexpr int N = 312, MM = 156;
    // eq. (step), w = 64: y = upper 33 bits of x_k | lower 31 of x_{k+1}
    static __device__ __forceinline__ W twist(W xk, W xk1, W xkm)
    {
        const uint32_t ylo = (lo32(xk) & 0x80000000u) | (lo32(xk1) & 0x7FFFFFFFu);
        const uint32_t yhi = hi32(xk);
        const uint32_t bit = lo32(xk1) & 1u;
        const uint32_t lo = lo32(xkm) ^ __funnelshift_r(ylo, yhi, 1) ^ (bit * 0xA96619E9u);
        const uint32_t hi = hi32(xkm) ^ (yhi >> 1) ^ (bit * 0xB5026F5Au);
        return pack64(lo, hi);
    }
    static __device__ __forceinline__ W twist(W xk, W xk1, W xkm, const ShiftK&) { return twist(xk, xk1, xkm); }
    // eq. (tempering), w = 64: (u, d, s, b, t, c, l) = (29, 5555555555555555,
    // 17, 71D67FFFEDA60000, 37, FFF7EEE000000000, 43)
    static __device__ __forceinline__ W temper(W y)
    {
        y ^= (y >> 29) & 0x5555555555555555ull;
        y ^= (y << 17) & 0x71D67FFFEDA60000ull;
        y ^= (y << 37) & 0xFFF7EEE000000000ull;
        return y ^ (y >> 43);
    }
    static __device__ __forceinline__ W temper(W y, const ShiftK& k)
    {
        uint32_t lo = lo32(y), hi = hi32(y);
        // y ^= (y >> 29) & d
        lo ^= __funnelshift_r(lo, hi, 29) & 0x55555555u;
        hi ^= (hi >> 29) & 0x55555555u;
        // y ^= (y << 17) & b
        const uint32_t th = __funnelshift_l(lo, hi, 17);
        lo ^= (lo * k.p17) & 0xEDA60000u;
        hi ^= th & 0x71D67FFFu;
        // y ^= (y << 37) & c: only the high half moves
        hi ^= (lo * k.p5) & 0xFFF7EEE0u;
        // y ^= y >> 43: only the low half changes
        lo ^= hi >> 11;
        return pack64(lo, hi);
    }
};

__device__ __constant__ static const uint32_t kSfmtMask[4] = {0xDFFFFFEFu, 0xDDFECB7Fu, 0xBFFAFFFFu, 0xBFFFFFF6u};

// ----------------------------------------------------------------------------
// conversions
// ----------------------------------------------------------------------------
__device__ __forceinline__ float f32_of_u32(uint32_t z) { return __uint2float_rz(z >> 8) * 5.9604644775390625e-8f; }

// exact double of v * 2^-53 for 0 <= v < 2^53, built from integer fields
__device__ __forceinline__ double f64_of_53(unsigned long long v)
{
    if (v == 0ull) return 0.0;
    const int sh = __clzll(v) - 11;  // leading one moved to bit 52
    const unsigned long long bits = (v << sh) + (static_cast<unsigned long long>(1021 - sh) << 52);
    return __longlong_as_double(static_cast<long long>(bits));
}

// the same for v = vh * 2^32 + vl (vh < 2^21) on 32-bit halves: when vh != 0
// (all but a 2^-21 share of the inputs) the leading one is in vh, so one
// 32-bit leading-zero count, one funnel shift and one shift normalise v, and
// the exponent 1021 - sh is added to the high half (the leading one at bit 52
// turns it into 1022 - sh, the exponent of a value in [2^-1-sh, 2^-sh))
__device__ __forceinline__ double f64_of_hilo(uint32_t vh, uint32_t vl)
{
    if (vh == 0u) return f64_of_53(vl);
    const int sh = __clz(vh) - 11;
    const uint32_t mh = __funnelshift_l(vl, vh, sh);
    const uint32_t ml = vl << sh;
    return __hiloint2double(static_cast<int>(mh + ((1021u - static_cast<uint32_t>(sh)) << 20)), static_cast<int>(ml));
}

__device__ __forceinline__ double f64_of_u64(unsigned long long z)
{
    return f64_of_hilo(hi32(z) >> 11, __funnelshift_r(lo32(z), hi32(z), 11));
}
// ((a >> 5) 2^26 + (b >> 6)) 2^-53: v = (a >> 11) 2^32 + (((a >> 5) << 26) | (b >> 6)) mod 2^32
__device__ __forceinline__ double f64_of_pair(uint32_t a, uint32_t b)
{
    return f64_of_hilo(a >> 11, ((a >> 5) << 26) | (b >> 6));
}
__device__ __forceinline__ float f32_of_u64(unsigned long long z) { return f32_of_u32(static_cast<uint32_t>(z >> 32)); }

// ----------------------------------------------------------------------------
// Emitter: routes word e (call-relative index in the V-stream) of one
// generator to its segment, converts it and stores it.  In lock-step launches
// generator g's outputs of segment s start at seg[s].out + g*seg[s].count
// elements; in unit launches the unit's single segment starts at unit_out.
// ----------------------------------------------------------------------------
__device__ __forceinline__ int elem_size(int dt) { return (dt == VMT_U32 || dt == VMT_F32) ? 4 : 8; }

struct Emitter {
    const GenArgs& a;
    long long g;      // generator index within the output arrays (lock-step)
    char* unit_out;   // unit mode: first output element of the unit, else nullptr

    // address of this generator's first output element of segment s
    __device__ __forceinline__ char* elem0(int s) const
    {
        if (unit_out) return unit_out;
        const SegArg& sg = a.seg[s];
        return sg.out + g * sg.count * elem_size(sg.dtype);
    }

    __device__ __forceinline__ int seg_of(long long e) const
    {
        int s = 0;
#pragma unroll
        for (int i = 1; i < VMT_MAXSEG; ++i)
            if (i < a.nseg && e >= a.seg[i].wbeg) s = i;
        return s;
    }

    // 32-bit words: z[0..VW) are words f0..f0+VW-1 of the block; the valid
    // block range is [lo, hi) and word f maps to e = ebase + f - lo.
    template <int VW>
    __device__ __forceinline__ void emit32(long long f0, const uint32_t (&z)[VW], long long lo, long long hi,
                                           long long ebase) const
    {
        const long long e0 = ebase + f0 - lo;
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            const long long f = f0 + u;
            if (f < lo || f >= hi) continue;
            const long long e = e0 + u;
            const int s = seg_of(e);
            const SegArg& sg = a.seg[s];
            const long long rel = e - sg.wbeg;
            char* base = elem0(s);
            switch (sg.dtype) {
            case VMT_U32: reinterpret_cast<uint32_t*>(base)[rel] = z[u]; break;
            case VMT_F32: reinterpret_cast<float*>(base)[rel] = f32_of_u32(z[u]); break;
            case VMT_U64:
                if ((rel & 1) == 0 && u + 1 < VW)
                    reinterpret_cast<unsigned long long*>(base)[rel / 2] =
                        static_cast<unsigned long long>(z[u]) | (static_cast<unsigned long long>(z[u + 1]) << 32);
                break;
            case VMT_F64:
                if ((rel & 1) == 0 && u + 1 < VW) reinterpret_cast<double*>(base)[rel / 2] = f64_of_pair(z[u], z[u + 1]);
                break;
            }
        }
    }

    // 64-bit words (MT19937-64): u64, f64 or f32 per word.
    template <int VW>
    __device__ __forceinline__ void emit64(long long f0, const unsigned long long (&z)[VW], long long lo,
                                           long long hi, long long ebase) const
    {
        const long long e0 = ebase + f0 - lo;
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            const long long f = f0 + u;
            if (f < lo || f >= hi) continue;
            const long long e = e0 + u;
            const int s = seg_of(e);
            const SegArg& sg = a.seg[s];
            const long long rel = e - sg.wbeg;
            char* base = elem0(s);
            switch (sg.dtype) {
            case VMT_U64: reinterpret_cast<unsigned long long*>(base)[rel] = z[u]; break;
            case VMT_F64: reinterpret_cast<double*>(base)[rel] = f64_of_u64(z[u]); break;
            case VMT_F32: reinterpret_cast<float*>(base)[rel] = f32_of_u64(z[u]); break;
            default: break;
            }
        }
    }
};

}  // namespace dev
}  // namespace vmt
