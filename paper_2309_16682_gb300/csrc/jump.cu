// jump.cu -- seeding, polynomial jump-ahead and the generic output conversion.
//
// Jump-ahead (Sec. 3.1): a lane is advanced by d steps as c(F) X with
// c = x^d mod mu.  For the generators here the state after i steps is the
// window (x_i, ..., x_{i+n-1}) of X's extended sequence x_0, x_1, ... (the
// circular buffer of eq. (staterec) never holds anything else), so
//
//     (c(F) X)_j = XOR over {i : c_i = 1} of x_{i+j},   j = 0..n-1.
//
// This is the Horner evaluation of c(F) X with the powers F^i X read off the
// sequence instead of recomputed, and it is parallel over j.  One warp owns
// one lane-jump: lane L accumulates output units j in [L R, L R + R) in
// registers and walks the coefficients of c in groups of R, reading each
// group's 2R-unit window of the sequence from a shared-memory ring that the
// warp extends with the recurrence ahead of the reads (n-m units at a time
// for MT, which are independent; one element at a time for SFMT, whose chain
// is serial).  Coefficients are taken two at a time so that one three-input
// XOR covers both when both are set.  The polynomial bits are uniform across
// the warp, so every branch is warp-uniform.
//
// Seeding (not in the paper): the C++ standard's mersenne_twister_engine
// initialisation (multiplier 1812433253 on 32-bit words, 6364136223846793005
// on 64-bit words); SFMT19937 fills its 624 32-bit sub-words with the 32-bit
// form and then applies its period certification with the parity vector
// (1, 0, 0, 0x13c9e684): when the parity of <p, w_0> is even the lowest set
// bit of p is flipped in w_0.
#include <atomic>

#include "vmt_device.cuh"
#include "vmt_internal.hpp"

namespace vmt {
namespace dev {

// ---------------------------------------------------------------------------
// seeding: one thread per generator, unit-major output base[u * count + g]
// ---------------------------------------------------------------------------
__global__ void seed_mt32_kernel(long long count, const unsigned long long* seeds, uint32_t* base)
{
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= count) return;
    uint32_t x = static_cast<uint32_t>(seeds[g]);
    base[g] = x;
    for (uint32_t i = 1; i < 624; ++i) {
        x = 1812433253u * (x ^ (x >> 30)) + i;
        base[static_cast<long long>(i) * count + g] = x;
    }
}

__global__ void seed_mt64_kernel(long long count, const unsigned long long* seeds, unsigned long long* base)
{
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= count) return;
    unsigned long long x = seeds[g];
    base[g] = x;
    for (unsigned long long i = 1; i < 312; ++i) {
        x = 6364136223846793005ull * (x ^ (x >> 62)) + i;
        base[static_cast<long long>(i) * count + g] = x;
    }
}

__global__ void seed_sfmt_kernel(long long count, const unsigned long long* seeds, uint4* base)
{
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= count) return;
    const uint32_t parity[4] = {0x00000001u, 0x00000000u, 0x00000000u, 0x13C9E684u};
    uint32_t x = static_cast<uint32_t>(seeds[g]);
    uint32_t e[4];
    e[0] = x;
    uint32_t i = 1;
    for (int k = 0; k < 156; ++k) {
        for (int s = (k == 0 ? 1 : 0); s < 4; ++s, ++i) {
            x = 1812433253u * (x ^ (x >> 30)) + i;
            e[s] = x;
        }
        if (k == 0) {
            // period certification on w_0
            uint32_t acc = (e[0] & parity[0]) ^ (e[1] & parity[1]) ^ (e[2] & parity[2]) ^ (e[3] & parity[3]);
            if ((__popc(acc) & 1) == 0) {
                bool done = false;
                for (int s = 0; s < 4 && !done; ++s)
                    for (int b = 0; b < 32 && !done; ++b)
                        if ((parity[s] >> b) & 1u) {
                            e[s] ^= 1u << b;
                            done = true;
                        }
            }
        }
        base[static_cast<long long>(k) * count + g] = make_uint4(e[0], e[1], e[2], e[3]);
    }
}

// ---------------------------------------------------------------------------
// jump kernel
// ---------------------------------------------------------------------------
constexpr int kJumpWarps = 4;

__device__ __forceinline__ uint32_t xor3(uint32_t a, uint32_t b, uint32_t c) { return a ^ b ^ c; }
__device__ __forceinline__ unsigned long long xor3(unsigned long long a, unsigned long long b, unsigned long long c)
{
    return a ^ b ^ c;
}
__device__ __forceinline__ uint4 xor3(uint4 a, uint4 b, uint4 c)
{
    return make_uint4(a.x ^ b.x ^ c.x, a.y ^ b.y ^ c.y, a.z ^ b.z ^ c.z, a.w ^ b.w ^ c.w);
}
__device__ __forceinline__ uint4 operator^(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }
template <typename U> __device__ __forceinline__ U zero_unit();
template <> __device__ __forceinline__ uint32_t zero_unit<uint32_t>() { return 0u; }
template <> __device__ __forceinline__ unsigned long long zero_unit<unsigned long long>() { return 0ull; }
template <> __device__ __forceinline__ uint4 zero_unit<uint4>() { return make_uint4(0u, 0u, 0u, 0u); }

// Jump configuration per generator: unit type U, n units, R outputs per
// lane, RING units of sequence per warp, C coefficients per refill.
struct JMT32 {
    using U = uint32_t;
    static constexpr int N = 624, MM = 397, R = 20, RING = 2560, C = 640, G = N - MM, PRE = 0;
};
struct JMT64 {
    using U = unsigned long long;
    static constexpr int N = 312, MM = 156, R = 10, RING = 1280, C = 320, G = N - MM, PRE = 0;
};
// SFMT: PRE units after the ring hold the chain-free parts of 32 new elements
struct JSFMT {
    using U = uint4;
    static constexpr int N = 156, MM = 122, R = 5, RING = 600, C = 160, G = 160, PRE = 32;
};

// SFMT19937 recurrence split in two: the part of w_q from w_{q-N} and
// w_{q-N+M}, which for 32 consecutive q only needs elements at least two
// places back and so can be computed in parallel, and the serial rest from
// w_{q-2} (128-bit right shift by 8) and w_{q-1} (32-bit left shifts by 18).
__device__ __forceinline__ uint4 sfmt_pre(uint4 a, uint4 b)
{
    uint4 p;
    p.x = a.x ^ (a.x << 8) ^ ((b.x >> 11) & kSfmtMask[0]);
    p.y = a.y ^ __funnelshift_l(a.x, a.y, 8) ^ ((b.y >> 11) & kSfmtMask[1]);
    p.z = a.z ^ __funnelshift_l(a.y, a.z, 8) ^ ((b.z >> 11) & kSfmtMask[2]);
    p.w = a.w ^ __funnelshift_l(a.z, a.w, 8) ^ ((b.w >> 11) & kSfmtMask[3]);
    return p;
}
__device__ __forceinline__ uint4 sfmt_chain(uint4 p, uint4 c, uint4 d)
{
    uint4 w;
    w.x = p.x ^ __funnelshift_r(c.x, c.y, 8) ^ (d.x << 18);
    w.y = p.y ^ __funnelshift_r(c.y, c.z, 8) ^ (d.y << 18);
    w.z = p.z ^ __funnelshift_r(c.z, c.w, 8) ^ (d.z << 18);
    w.w = p.w ^ (c.w >> 8) ^ (d.w << 18);
    return w;
}

// One thread runs the chain through n <= 32 elements whose chain-free parts
// are pre[0..n), writing them to ring[iq], ring[iq + 1], ... (modulo RG);
// c and d are w_{q-2} and w_{q-1} and are carried on.  The parts are read
// eight at a time ahead of the chain (the compiler cannot move a read of pre
// above a write of the ring, which it must assume may alias).
template <int RG>
__device__ __forceinline__ void sfmt_chain_run(const uint4* pre, uint4* ring, int iq, int n, uint4& c, uint4& d)
{
    for (int u0 = 0; u0 < n; u0 += 8) {
        uint4 p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = pre[u0 + k];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (u0 + k < n) {
                const uint4 w = sfmt_chain(p[k], c, d);
                ring[iq] = w;
                iq = iq + 1 == RG ? 0 : iq + 1;
                c = d;
                d = w;
            }
        }
    }
}

// extend the sequence: units [gen, gen + G) of the ring (the grid carries the
// recurrence of run-time generators)
template <class J>
__device__ __forceinline__ void extend(typename J::U* ring, int gen, int lane, const JumpGrid& gr);

template <>
__device__ __forceinline__ void extend<JMT32>(uint32_t* ring, int gen, int lane, const JumpGrid&)
{
    constexpr int RG = JMT32::RING;
    for (int u = lane; u < JMT32::G; u += 32) {
        const int k = gen - JMT32::N + u;
        ring[(gen + u) % RG] = MT32::twist(ring[k % RG], ring[(k + 1) % RG], ring[(k + JMT32::MM) % RG]);
    }
}

template <>
__device__ __forceinline__ void extend<JMT64>(unsigned long long* ring, int gen, int lane, const JumpGrid&)
{
    constexpr int RG = JMT64::RING;
    for (int u = lane; u < JMT64::G; u += 32) {
        const int k = gen - JMT64::N + u;
        ring[(gen + u) % RG] = MT64::twist(ring[k % RG], ring[(k + 1) % RG], ring[(k + JMT64::MM) % RG]);
    }
}

template <>
__device__ __forceinline__ void extend<JSFMT>(uint4* ring, int gen, int lane, const JumpGrid&)
{
    // 32 elements at a time: every lane the chain-free part of one element,
    // then four lanes the chain through all 32
    constexpr int RG = JSFMT::RING, NN = JSFMT::N, MMM = JSFMT::MM;
    static_assert(JSFMT::G % 32 == 0 && NN - MMM >= 32, "blocks of 32 elements");
    uint4* pre = ring + RG;
    for (int s0 = gen; s0 < gen + JSFMT::G; s0 += 32) {
        const int q = s0 + lane;
        pre[lane] = sfmt_pre(ring[(q - NN) % RG], ring[(q - NN + MMM) % RG]);
        __syncwarp();
        if (lane < 4) {
            // lanes 0..3 run the chain, lane j owning sub-word j; the 128-bit
            // right shift of w_{q-2} takes sub-word j+1 from the next lane,
            // passed one step ahead of its use
            const uint32_t* p32 = reinterpret_cast<const uint32_t*>(pre);
            uint32_t* r32 = reinterpret_cast<uint32_t*>(ring);
            uint32_t c = r32[4 * ((s0 - 2) % RG) + lane], d = r32[4 * ((s0 - 1) % RG) + lane];
            uint32_t cn = __shfl_down_sync(0xFu, c, 1, 4);
            if (lane == 3) cn = 0u;
            int iq = s0 % RG;
#pragma unroll 8
            for (int u = 0; u < 32; ++u) {
                const uint32_t w = p32[4 * u + lane] ^ __funnelshift_r(c, cn, 8) ^ (d << 18);
                r32[4 * iq + lane] = w;
                const uint32_t dn = __shfl_down_sync(0xFu, d, 1, 4);
                iq = iq + 1 == RG ? 0 : iq + 1;
                c = d;
                cn = lane == 3 ? 0u : dn;
                d = w;
            }
        }
        __syncwarp();
    }
}

template <typename U>
__device__ __forceinline__ U ld_unit(const void* base, long long idx)
{
    return reinterpret_cast<const U*>(base)[idx];
}

// R consecutive units starting at ring index rb (a multiple of R, so the group
// never wraps and is 16-byte aligned), as 16-byte shared-memory loads.
template <class J>
__device__ __forceinline__ void load_group(const typename J::U* ring, int rb, typename J::U (&w)[J::R])
{
    using U = typename J::U;
    constexpr int V = J::R * static_cast<int>(sizeof(U)) / 16;
    const uint4* p = reinterpret_cast<const uint4*>(ring + rb);
    uint4 t[V];
#pragma unroll
    for (int v = 0; v < V; ++v) t[v] = p[v];
    memcpy(w, t, sizeof(t));
}

template <class J, int S, int R>
struct Win {
    // unit s + r of the 2R-unit window held as wA | wB
    template <typename U>
    static __device__ __forceinline__ U get(const U (&wA)[R], const U (&wB)[R], int r)
    {
        return (S + r < R) ? wA[(S + r < R) ? S + r : 0] : wB[(S + r >= R) ? S + r - R : 0];
    }
};

template <class J, int S>
__device__ __forceinline__ void apply_pair(uint32_t bits, typename J::U (&acc)[J::R], const typename J::U (&wA)[J::R],
                                           const typename J::U (&wB)[J::R])
{
    constexpr int R = J::R;
    const uint32_t b2 = (bits >> S) & 3u;
    if (S + 1 < R && b2 == 3u) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = xor3(acc[r], Win<J, S, R>::get(wA, wB, r), Win<J, S + 1, R>::get(wA, wB, r));
    } else if (b2 & 1u) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = acc[r] ^ Win<J, S, R>::get(wA, wB, r);
    } else if (S + 1 < R && (b2 & 2u)) {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = acc[r] ^ Win<J, S + 1, R>::get(wA, wB, r);
    }
}

template <class J, int S>
struct ApplyAll {
    static __device__ __forceinline__ void run(uint32_t bits, typename J::U (&acc)[J::R], const typename J::U (&wA)[J::R],
                                               const typename J::U (&wB)[J::R])
    {
        apply_pair<J, S>(bits, acc, wA, wB);
        ApplyAll<J, S + 2>::run(bits, acc, wA, wB);
    }
};
template <class J> struct ApplyAll<J, J::R> {
    static __device__ __forceinline__ void run(uint32_t, typename J::U (&)[J::R], const typename J::U (&)[J::R],
                                               const typename J::U (&)[J::R]) {}
};
template <class J> struct ApplyAll<J, J::R + 1> {
    static __device__ __forceinline__ void run(uint32_t, typename J::U (&)[J::R], const typename J::U (&)[J::R],
                                               const typename J::U (&)[J::R]) {}
};

// Work item `item` of a grid description (see JumpGrid); false when the item
// has nothing to do (a zero digit).
__device__ __forceinline__ bool grid_item(const JumpGrid& gr, long long item, JumpItem& it)
{
    if (gr.mode == JumpGrid::kFanOut) {
        const long long g = item / gr.lanes;
        const int t = static_cast<int>(item % gr.lanes);
        it.src = gr.base + g * gr.unit_bytes;
        it.src_stride = static_cast<int>(gr.count);
        it.dst = gr.states + g * gr.gen_bytes + static_cast<long long>(t) * gr.unit_bytes;
        it.dst_stride = gr.lanes;
        it.poly = t * 16 / gr.lanes;
    } else if (gr.mode == JumpGrid::kChunk) {
        const long long k = item / gr.lanes;
        const int t = static_cast<int>(item % gr.lanes);
        const int2 rc = gr.chunk_map[k];
        it.src = gr.base + static_cast<long long>(rc.x) * gr.gen_bytes + static_cast<long long>(t) * gr.unit_bytes;
        it.src_stride = gr.lanes;
        it.dst = gr.states + k * gr.gen_bytes + static_cast<long long>(t) * gr.unit_bytes;
        it.dst_stride = gr.lanes;
        it.poly = gr.chunk_row0 + rc.y - 1;
    } else {
        const long long g = item;
        const int dig = static_cast<int>((gr.jumps[g] >> (8 * gr.digit)) & 255u);
        if (dig == 0) return false;
        it.src = gr.base + g * gr.unit_bytes;
        it.dst = gr.base + g * gr.unit_bytes;
        it.src_stride = static_cast<int>(gr.count);
        it.dst_stride = static_cast<int>(gr.count);
        it.poly = 16 + 255 * gr.digit + dig - 1;
    }
    it.deg = gr.row_deg[it.poly];
    return true;
}

template <class J>
__global__ void __launch_bounds__(kJumpWarps * 32) jump_kernel(const JumpItem* items, JumpGrid grid,
                                                                long long nitems, const uint32_t* polys)
{
    using U = typename J::U;
    constexpr int N = J::N, R = J::R, RING = J::RING, C = J::C;
    static_assert(RING % R == 0 && C % R == 0, "groups must not wrap the ring");
    static_assert(RING >= C + 32 * R + J::G && RING >= N + J::G, "ring too small");
    __shared__ __align__(16) U ring_all[kJumpWarps][RING + J::PRE];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long item = static_cast<long long>(blockIdx.x) * kJumpWarps + warp;
    if (item >= nitems) return;  // whole warp leaves together
    JumpItem it;
    if (items) it = items[item];
    else if (!grid_item(grid, item, it)) return;
    U* ring = ring_all[warp];
    for (int u = lane; u < N; u += 32) ring[u] = ld_unit<U>(it.src, static_cast<long long>(u) * it.src_stride);
    __syncwarp();

    const uint32_t* c = polys + static_cast<long long>(it.poly) * kPolyWords;
    const int deg = it.deg;
    const int j0 = lane * R;
    U acc[R], wA[R], wB[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = zero_unit<U>();

    int gen = N;
    for (int i0 = 0; i0 <= deg; i0 += C) {
        const int need = i0 + C + 32 * R;
        while (gen < need) {
            extend<J>(ring, gen, lane, grid);
            gen += J::G;
            __syncwarp();
        }
        if (i0 == 0) load_group<J>(ring, j0 % RING, wA);
        const int iend = min(i0 + C, deg + 1);
        for (int ib = i0; ib < iend; ib += R) {
            load_group<J>(ring, (ib + R + j0) % RING, wB);
            const int wi = ib >> 5, sh = ib & 31;
            const unsigned long long two = static_cast<unsigned long long>(__ldg(c + wi)) |
                                           (static_cast<unsigned long long>(__ldg(c + wi + 1)) << 32);
            const uint32_t bits = static_cast<uint32_t>(two >> sh) & ((1u << R) - 1u);
            if (bits) ApplyAll<J, 0>::run(bits, acc, wA, wB);
#pragma unroll
            for (int r = 0; r < R; ++r) wA[r] = wB[r];
        }
    }
    U* dst = reinterpret_cast<U*>(it.dst);
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (j0 + r < N) dst[static_cast<long long>(j0 + r) * it.dst_stride] = acc[r];
}

// ---------------------------------------------------------------------------
// jump kernel for small launches: one CTA per lane-jump
// ---------------------------------------------------------------------------
// The same evaluation with one lane-jump spread over the W warps of a CTA by
// splitting the coefficients of c: the CTA extends the sequence into a large
// shared ring (the whole extended sequence for MT19937-32/64, two rounds for
// SFMT19937), warp w walks the w-th slice of the round's coefficients exactly
// as one warp of jump_kernel walks all of them (lane L holding output units
// [L R, L R + R)), and at the end the W partial results are XORed.  A
// lane-jump costs about as many instructions as in jump_kernel, but its
// latency is W times shorter, which is what launches of a few hundred items
// (a batch of requests, the lanes of a few generators) are bound by.
struct CMT32 {
    using U = uint32_t;
    static constexpr int N = 624, MM = 397, G = N - MM, R = 20, W = 16, L = 21120, PRE = 0;
};
struct CMT64 {
    using U = unsigned long long;
    static constexpr int N = 312, MM = 156, G = N - MM, R = 10, W = 16, L = 20760, PRE = 0;
};
struct CSFMT {
    using U = uint4;
    static constexpr int N = 156, MM = 122, G = 0, R = 5, W = 16, L = 12000, PRE = 32;
};
// Compact forms: four warps over a ring of about 20 KB, the sequence extended
// in several rounds.  A lane-jump takes about four times longer than in the
// sixteen-warp form, but a CTA needs little shared memory, so it finds an SM
// next to running generation CTAs (the server's initialisation).
struct CMT32C {
    using U = uint32_t;
    static constexpr int N = 624, MM = 397, G = N - MM, R = 20, W = 4, L = 5120, PRE = 0;
};
struct CMT64C {
    using U = unsigned long long;
    static constexpr int N = 312, MM = 156, G = N - MM, R = 10, W = 4, L = 2560, PRE = 0;
};
struct CSFMTC {
    using U = uint4;
    static constexpr int N = 156, MM = 122, G = 0, R = 5, W = 4, L = 1280, PRE = 32;
};
// coefficients per round: the ring holds the round's window of C + 33 R units
// plus one extension step
template <class S> __host__ __device__ constexpr int cta_round() { return (S::L - 33 * S::R - S::G) / (S::R * S::W) * (S::R * S::W); }
template <class S> __host__ __device__ constexpr size_t cta_smem()
{
    return static_cast<size_t>(S::L + S::PRE) * sizeof(typename S::U);
}

__device__ __forceinline__ int wrap_sub(int p, int L) { return p >= L ? p - L : p; }

// extend the ring from unit gen up to (at least) unit need; every thread
// calls it with the same arguments and gets the same new gen
template <class S>
__device__ __forceinline__ int cta_extend(typename S::U* ring, int gen, int need, int tid, const JumpGrid& gr);

template <class S, class T>
__device__ __forceinline__ int cta_extend_mt(typename S::U* ring, int gen, int need, int tid)
{
    constexpr int L = S::L;
    while (gen < need) {
        // the G new words of a step are independent; a CTA may have fewer threads
        for (int u = tid; u < S::G; u += S::W * 32) {
            const int q = gen + u;   // ring positions are taken modulo L
            const int k = (q - S::N) % L;
            ring[q % L] = T::twist(ring[k], ring[wrap_sub(k + 1, L)], ring[wrap_sub(k + S::MM, L)]);
        }
        gen += S::G;
        __syncthreads();
    }
    return gen;
}
template <>
__device__ __forceinline__ int cta_extend<CMT32>(uint32_t* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_mt<CMT32, MT32>(ring, gen, need, tid);
}
template <>
__device__ __forceinline__ int cta_extend<CMT64>(unsigned long long* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_mt<CMT64, MT64>(ring, gen, need, tid);
}
template <>
__device__ __forceinline__ int cta_extend<CMT32C>(uint32_t* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_mt<CMT32C, MT32>(ring, gen, need, tid);
}
template <>
__device__ __forceinline__ int cta_extend<CMT64C>(unsigned long long* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_mt<CMT64C, MT64>(ring, gen, need, tid);
}
// SFMT: 32 elements at a time, warp 1 computing their chain-free parts into
// the 32 units after the ring and thread 0 running the chain through them;
// the two warps meet at named barrier 1, the other warps wait at the end
template <class S>
__device__ __forceinline__ int cta_extend_sfmt(uint4* ring, int gen, int need, int tid)
{
    constexpr int L = S::L, NN = S::N, MMM = S::MM;
    static_assert(NN - MMM >= 32 && S::W >= 2, "blocks of 32 elements, two warps");
    uint4* pre = ring + L;
    if (tid < 64) {
        uint4 c = make_uint4(0u, 0u, 0u, 0u), d = c;
        if (tid == 0 && gen < need) {
            c = ring[(gen - 2) % L];
            d = ring[(gen - 1) % L];
        }
        for (int s0 = gen; s0 < need; s0 += 32) {
            const int cnt = min(32, need - s0);
            const int lane = tid - 32;
            if (lane >= 0 && lane < cnt) {
                const int q = s0 + lane;
                pre[lane] = sfmt_pre(ring[(q - NN) % L], ring[(q - NN + MMM) % L]);
            }
            asm volatile("bar.sync 1, 64;" ::: "memory");
            if (tid == 0) {
                if (cnt == 32) sfmt_chain_run<L>(pre, ring, s0 % L, 32, c, d);   // full blocks: no predication
                else sfmt_chain_run<L>(pre, ring, s0 % L, cnt, c, d);
            }
            asm volatile("bar.sync 1, 64;" ::: "memory");
        }
    }
    __syncthreads();
    return need > gen ? need : gen;
}
template <>
__device__ __forceinline__ int cta_extend<CSFMT>(uint4* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_sfmt<CSFMT>(ring, gen, need, tid);
}
template <>
__device__ __forceinline__ int cta_extend<CSFMTC>(uint4* ring, int gen, int need, int tid, const JumpGrid&)
{
    return cta_extend_sfmt<CSFMTC>(ring, gen, need, tid);
}

template <class S>
__global__ void __launch_bounds__(S::W * 32) jump_cta_kernel(const JumpItem* items, JumpGrid grid, const uint32_t* polys)
{
    using U = typename S::U;
    constexpr int N = S::N, R = S::R, W = S::W, L = S::L, C = cta_round<S>();
    static_assert(L % R == 0 && R * sizeof(U) % 16 == 0, "R-unit groups are aligned 16-byte loads that never wrap");
    static_assert(C > 0 && L >= C + 33 * R + S::G && L >= N + S::G, "ring too small");
    static_assert(W * 32 * R <= L && 32 * R >= N, "partial results must fit the ring");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    U* ring = reinterpret_cast<U*>(smem_raw);
    const long long item = blockIdx.x;
    JumpItem it;
    if (items) it = items[item];
    else if (!grid_item(grid, item, it)) return;   // the same answer for every thread
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int u = tid; u < N; u += W * 32) ring[u] = ld_unit<U>(it.src, static_cast<long long>(u) * it.src_stride);
    __syncthreads();

    const uint32_t* c = polys + static_cast<long long>(it.poly) * kPolyWords;
    const int deg = it.deg;
    const int j0 = lane * R;
    U acc[R], wA[R], wB[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = zero_unit<U>();
    int gen = N;
    for (int i0 = 0; i0 <= deg; i0 += C) {
        const int iend = min(i0 + C, deg + 1);
        gen = cta_extend<S>(ring, gen, iend + 33 * R, tid, grid);
        // this warp's slice of the round's coefficients, a multiple of R long
        const int span = ((iend - i0 + W * R - 1) / (W * R)) * R;
        const int lo = i0 + warp * span, hi = min(lo + span, iend);
        if (lo < hi) {
            load_group<S>(ring, (lo + j0) % L, wA);
            for (int ib = lo; ib < hi; ib += R) {
                load_group<S>(ring, (ib + R + j0) % L, wB);
                const int wi = ib >> 5, sh = ib & 31;
                const unsigned long long two = static_cast<unsigned long long>(__ldg(c + wi)) |
                                               (static_cast<unsigned long long>(__ldg(c + wi + 1)) << 32);
                const uint32_t bits = static_cast<uint32_t>(two >> sh) & ((1u << R) - 1u);
                if (bits) ApplyAll<S, 0>::run(bits, acc, wA, wB);
#pragma unroll
                for (int r = 0; r < R; ++r) wA[r] = wB[r];
            }
        }
        __syncthreads();   // the round is consumed before the ring moves on
    }
    // XOR of the W partial results
#pragma unroll
    for (int r = 0; r < R; ++r) ring[warp * 32 * R + j0 + r] = acc[r];
    __syncthreads();
    U* dst = reinterpret_cast<U*>(it.dst);
    for (int j = tid; j < N; j += W * 32) {
        U x = ring[j];
#pragma unroll
        for (int w = 1; w < W; ++w) x = x ^ ring[w * 32 * R + j];
        dst[static_cast<long long>(j) * it.dst_stride] = x;
    }
}

// ---------------------------------------------------------------------------
// twisted GFSR with run-time parameters (w <= 32, compiled n): the same
// window-correlation kernels, with the sequence extended one word at a time
// by the recurrence the grid carries.  Used to check the jump kernels on
// generators small enough for the matrix route of Sec. 3.1, and for F2-linear
// generators other than the three above.
// ---------------------------------------------------------------------------
template <int N_>
struct JTG {
    using U = uint32_t;
    static constexpr int N = N_, MM = 1, R = 4, RING = 260, C = 128, G = 1, PRE = 0;
};
template <int N_>
struct CTG {
    using U = uint32_t;
    static constexpr int N = N_, MM = 1, G = 1, R = 4, W = 4, L = 1024, PRE = 0;
};

__device__ __forceinline__ uint32_t tg_twist(uint32_t xk, uint32_t xk1, uint32_t xkm, const JumpGrid& g)
{
    const uint32_t y = (xk & g.tg_upper) | (xk1 & g.tg_lower);
    return xkm ^ (y >> 1) ^ ((y & 1u) ? g.tg_a : 0u);
}

// one new word (lane 0) per call; the kernel's __syncwarp follows
template <int N_>
__device__ __forceinline__ void extend_tg(uint32_t* ring, int gen, int lane, const JumpGrid& g)
{
    constexpr int RG = JTG<N_>::RING;
    if (lane == 0) {
        const int k = gen - N_;
        ring[gen % RG] = tg_twist(ring[k % RG], ring[(k + 1) % RG], ring[(k + static_cast<int>(g.tg_m)) % RG], g);
    }
}
template <> __device__ __forceinline__ void extend<JTG<4>>(uint32_t* r, int gen, int lane, const JumpGrid& g) { extend_tg<4>(r, gen, lane, g); }
template <> __device__ __forceinline__ void extend<JTG<5>>(uint32_t* r, int gen, int lane, const JumpGrid& g) { extend_tg<5>(r, gen, lane, g); }
template <> __device__ __forceinline__ void extend<JTG<17>>(uint32_t* r, int gen, int lane, const JumpGrid& g) { extend_tg<17>(r, gen, lane, g); }

template <int N_>
__device__ __forceinline__ int cta_extend_tg(uint32_t* ring, int gen, int need, int tid, const JumpGrid& g)
{
    constexpr int L = CTG<N_>::L;
    for (; gen < need; ++gen) {
        if (tid == 0) {
            const int k = gen - N_;
            ring[gen % L] = tg_twist(ring[k % L], ring[(k + 1) % L], ring[(k + static_cast<int>(g.tg_m)) % L], g);
        }
        __syncthreads();
    }
    return gen;
}
template <> __device__ __forceinline__ int cta_extend<CTG<4>>(uint32_t* r, int gen, int need, int tid, const JumpGrid& g) { return cta_extend_tg<4>(r, gen, need, tid, g); }
template <> __device__ __forceinline__ int cta_extend<CTG<5>>(uint32_t* r, int gen, int need, int tid, const JumpGrid& g) { return cta_extend_tg<5>(r, gen, need, tid, g); }
template <> __device__ __forceinline__ int cta_extend<CTG<17>>(uint32_t* r, int gen, int need, int tid, const JumpGrid& g) { return cta_extend_tg<17>(r, gen, need, tid, g); }

// Launches of fewer items than this use the CTA-per-item kernel, per variant
// (the crossover in lane-jumps per second measured on GB300: about 4096 for
// MT19937-32/64, about 512 for SFMT19937, whose serial chain makes the CTA
// kernel's lane-jump long).
static std::atomic<long long> g_split_below[3] = {{4096}, {4096}, {512}};
// every launch of the variant in the compact CTA form (callers that share the
// GPU with long-running kernels; tests)
static std::atomic<int> g_compact[3] = {{0}, {0}, {0}};

// the CTA kernels' dynamic shared memory limit, raised once per device
template <class S>
static cudaError_t cta_smem_attr()
{
    constexpr int kMaxDev = 64;
    static std::atomic<bool> done[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDev && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(jump_cta_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(cta_smem<S>()));
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDev) done[dev].store(true, std::memory_order_release);
    return e;
}

template <class S>
static cudaError_t launch_cta_form(const JumpItem* items, const JumpGrid& gr, long long nitems, const uint32_t* polys,
                                   cudaStream_t st)
{
    const cudaError_t e = cta_smem_attr<S>();
    if (e != cudaSuccess) return e;
    jump_cta_kernel<S><<<static_cast<unsigned>(nitems), S::W * 32, cta_smem<S>(), st>>>(items, gr, polys);
    return cudaGetLastError();
}

// shared: 0 the default choice (sixteen-warp CTA or warp kernel by count),
// 1 compact CTAs (for launches that share the GPU)
template <class J, class S, class SC>
static cudaError_t launch_jump_t(int variant, const JumpItem* items, const JumpGrid& gr, long long nitems,
                                 const uint32_t* polys, cudaStream_t st, long long split_below, int shared)
{
    if (nitems <= 0) return cudaSuccess;
    const int forced = g_compact[variant].load(std::memory_order_relaxed);
    const int form = shared ? shared : forced;
    if (form == 1) return launch_cta_form<SC>(items, gr, nitems, polys, st);
    if (nitems < split_below) {
        const cudaError_t e = cta_smem_attr<S>();
        if (e != cudaSuccess) return e;
        jump_cta_kernel<S><<<static_cast<unsigned>(nitems), S::W * 32, cta_smem<S>(), st>>>(items, gr, polys);
        return cudaGetLastError();
    }
    const long long grid = (nitems + kJumpWarps - 1) / kJumpWarps;
    jump_kernel<J><<<static_cast<unsigned>(grid), kJumpWarps * 32, 0, st>>>(items, gr, nitems, polys);
    return cudaGetLastError();
}

__global__ void fill_int_kernel(int* p, long long n, int v)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// generic conversion: native words (u32 or u64) of each generator, laid out
// [g][words], are converted into one output segment; used when a segment's
// alignment rules out the fused path (odd word offset of a two-word type).
// ---------------------------------------------------------------------------
__global__ void convert_kernel(const void* words, long long words_per_gen, int word64, long long gens, long long wbeg,
                               int dtype, long long count, void* out)
{
    const long long total = gens * count;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const long long g = i / count, o = i % count;
        if (word64) {
            const unsigned long long z = reinterpret_cast<const unsigned long long*>(words)[g * words_per_gen + wbeg + o];
            if (dtype == VMT_U64) reinterpret_cast<unsigned long long*>(out)[i] = z;
            else if (dtype == VMT_F64) reinterpret_cast<double*>(out)[i] = f64_of_u64(z);
            else reinterpret_cast<float*>(out)[i] = f32_of_u64(z);
        } else {
            const uint32_t* w = reinterpret_cast<const uint32_t*>(words) + g * words_per_gen + wbeg;
            if (dtype == VMT_U32) reinterpret_cast<uint32_t*>(out)[i] = w[o];
            else if (dtype == VMT_F32) reinterpret_cast<float*>(out)[i] = f32_of_u32(w[o]);
            else if (dtype == VMT_U64)
                reinterpret_cast<unsigned long long*>(out)[i] =
                    static_cast<unsigned long long>(w[2 * o]) | (static_cast<unsigned long long>(w[2 * o + 1]) << 32);
            else reinterpret_cast<double*>(out)[i] = f64_of_pair(w[2 * o], w[2 * o + 1]);
        }
    }
}

}  // namespace dev

cudaError_t launch_seed(int variant, long long count, const unsigned long long* seeds, void* base, cudaStream_t s)
{
    using namespace dev;
    if (count <= 0) return cudaSuccess;
    const int T = 128;
    const unsigned grid = static_cast<unsigned>((count + T - 1) / T);
    if (variant == VMT_MT19937_32) seed_mt32_kernel<<<grid, T, 0, s>>>(count, seeds, static_cast<uint32_t*>(base));
    else if (variant == VMT_MT19937_64)
        seed_mt64_kernel<<<grid, T, 0, s>>>(count, seeds, static_cast<unsigned long long*>(base));
    else seed_sfmt_kernel<<<grid, T, 0, s>>>(count, seeds, static_cast<uint4*>(base));
    return cudaGetLastError();
}

cudaError_t launch_jump(int variant, const JumpItem* items, long long nitems, const uint32_t* polys, cudaStream_t s,
                        int compact)
{
    using namespace dev;
    if (variant < 0 || variant > 2) return cudaErrorInvalidValue;
    const JumpGrid none{};
    const long long sb = g_split_below[variant].load(std::memory_order_relaxed);
    if (variant == VMT_MT19937_32) return launch_jump_t<JMT32, CMT32, CMT32C>(variant, items, none, nitems, polys, s, sb, compact);
    if (variant == VMT_MT19937_64) return launch_jump_t<JMT64, CMT64, CMT64C>(variant, items, none, nitems, polys, s, sb, compact);
    return launch_jump_t<JSFMT, CSFMT, CSFMTC>(variant, items, none, nitems, polys, s, sb, compact);
}

cudaError_t launch_jump_grid(int variant, const JumpGrid& gr, long long nitems, const uint32_t* polys, cudaStream_t s,
                             int compact)
{
    using namespace dev;
    if (variant < 0 || variant > 2) return cudaErrorInvalidValue;
    const long long sb = g_split_below[variant].load(std::memory_order_relaxed);
    if (variant == VMT_MT19937_32) return launch_jump_t<JMT32, CMT32, CMT32C>(variant, nullptr, gr, nitems, polys, s, sb, compact);
    if (variant == VMT_MT19937_64) return launch_jump_t<JMT64, CMT64, CMT64C>(variant, nullptr, gr, nitems, polys, s, sb, compact);
    return launch_jump_t<JSFMT, CSFMT, CSFMTC>(variant, nullptr, gr, nitems, polys, s, sb, compact);
}

namespace dev {
template <int N>
static cudaError_t launch_tg_n(bool cta, const JumpItem* items, long long nitems, const JumpGrid& gr,
                               const uint32_t* polys, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (cta) {
        const cudaError_t e = cta_smem_attr<CTG<N>>();
        if (e != cudaSuccess) return e;
        jump_cta_kernel<CTG<N>><<<static_cast<unsigned>(nitems), CTG<N>::W * 32, cta_smem<CTG<N>>(), st>>>(items, gr,
                                                                                                          polys);
    } else {
        const long long grid = (nitems + kJumpWarps - 1) / kJumpWarps;
        jump_kernel<JTG<N>><<<static_cast<unsigned>(grid), kJumpWarps * 32, 0, st>>>(items, gr, nitems, polys);
    }
    return cudaGetLastError();
}
}  // namespace dev

cudaError_t launch_tgfsr_jump(int n, bool cta, const JumpItem* items, long long nitems, const JumpGrid& gr,
                              const uint32_t* polys, cudaStream_t s)
{
    switch (n) {
    case 4: return dev::launch_tg_n<4>(cta, items, nitems, gr, polys, s);
    case 5: return dev::launch_tg_n<5>(cta, items, nitems, gr, polys, s);
    case 17: return dev::launch_tg_n<17>(cta, items, nitems, gr, polys, s);
    }
    return cudaErrorNotSupported;
}

void set_jump_split_below(int variant, long long items) { dev::g_split_below[variant].store(items < 0 ? 0 : items); }
void set_jump_compact(int variant, int form) { dev::g_compact[variant].store(form); }
int get_jump_compact(int variant) { return dev::g_compact[variant].load(); }
long long get_jump_split_below(int variant) { return dev::g_split_below[variant].load(); }

cudaError_t launch_fill_int(int* p, long long n, int value, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    dev::fill_int_kernel<<<static_cast<unsigned>(grid), 256, 0, s>>>(p, n, value);
    return cudaGetLastError();
}

cudaError_t launch_convert(const void* words, long long words_per_gen, int word64, long long gens, long long wbeg,
                           int dtype, long long count, void* out, cudaStream_t s)
{
    const long long total = gens * count;
    if (total <= 0) return cudaSuccess;
    const int T = 256;
    long long grid = (total + T - 1) / T;
    if (grid > 152LL * 64) grid = 152LL * 64;
    dev::convert_kernel<<<static_cast<unsigned>(grid), T, 0, s>>>(words, words_per_gen, word64, gens, wbeg, dtype,
                                                                   count, out);
    return cudaGetLastError();
}

}  // namespace vmt
