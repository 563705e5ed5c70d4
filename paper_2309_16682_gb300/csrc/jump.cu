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
#include "vmt_device.cuh"

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
    static constexpr int N = 624, MM = 397, R = 20, RING = 2560, C = 640, G = N - MM;
};
struct JMT64 {
    using U = unsigned long long;
    static constexpr int N = 312, MM = 156, R = 10, RING = 1280, C = 320, G = N - MM;
};
struct JSFMT {
    using U = uint4;
    static constexpr int N = 156, MM = 122, R = 5, RING = 640, C = 160, G = 160;
};

// extend the sequence: units [gen, gen + G) of the ring
template <class J>
__device__ __forceinline__ void extend(typename J::U* ring, int gen, int lane);

template <>
__device__ __forceinline__ void extend<JMT32>(uint32_t* ring, int gen, int lane)
{
    constexpr int RG = JMT32::RING;
    for (int u = lane; u < JMT32::G; u += 32) {
        const int k = gen - JMT32::N + u;
        ring[(gen + u) % RG] = MT32::twist(ring[k % RG], ring[(k + 1) % RG], ring[(k + JMT32::MM) % RG]);
    }
}

template <>
__device__ __forceinline__ void extend<JMT64>(unsigned long long* ring, int gen, int lane)
{
    constexpr int RG = JMT64::RING;
    for (int u = lane; u < JMT64::G; u += 32) {
        const int k = gen - JMT64::N + u;
        ring[(gen + u) % RG] = MT64::twist(ring[k % RG], ring[(k + 1) % RG], ring[(k + JMT64::MM) % RG]);
    }
}

template <>
__device__ __forceinline__ void extend<JSFMT>(uint4* ring, int gen, int lane)
{
    // four lanes, one 32-bit sub-word each; serial over the G new elements
    constexpr int RG = JSFMT::RING, NN = JSFMT::N, MMM = JSFMT::MM;
    if (lane >= 4) return;
    const int j = lane;
    const uint32_t K = kSfmtMask[j];
    uint32_t* r32 = reinterpret_cast<uint32_t*>(ring);
    uint32_t d = r32[4 * ((gen - 1) % RG) + j];   // w_{q-1}
    uint32_t c = r32[4 * ((gen - 2) % RG) + j];   // w_{q-2}
    for (int u = 0; u < JSFMT::G; ++u) {
        const int q = gen + u;
        const uint32_t wa = r32[4 * ((q - NN) % RG) + j];
        const uint32_t wb = r32[4 * ((q - NN + MMM) % RG) + j];
        uint32_t am1 = __shfl_up_sync(0xFu, wa, 1, 4);
        uint32_t cp1 = __shfl_down_sync(0xFu, c, 1, 4);
        if (j == 0) am1 = 0u;
        if (j == 3) cp1 = 0u;
        const uint32_t nw = wa ^ __funnelshift_l(am1, wa, 8) ^ ((wb >> 11) & K) ^ __funnelshift_r(c, cp1, 8) ^ (d << 18);
        r32[4 * (q % RG) + j] = nw;
        c = d;
        d = nw;
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
    __shared__ __align__(16) U ring_all[kJumpWarps][RING];
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
            extend<J>(ring, gen, lane);
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

template <class J>
static cudaError_t launch_jump_t(const JumpItem* items, const JumpGrid& gr, long long nitems, const uint32_t* polys,
                                 cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
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

cudaError_t launch_jump(int variant, const JumpItem* items, long long nitems, const uint32_t* polys, cudaStream_t s)
{
    using namespace dev;
    const JumpGrid none{};
    if (variant == VMT_MT19937_32) return launch_jump_t<JMT32>(items, none, nitems, polys, s);
    if (variant == VMT_MT19937_64) return launch_jump_t<JMT64>(items, none, nitems, polys, s);
    return launch_jump_t<JSFMT>(items, none, nitems, polys, s);
}

cudaError_t launch_jump_grid(int variant, const JumpGrid& gr, long long nitems, const uint32_t* polys, cudaStream_t s)
{
    using namespace dev;
    if (variant == VMT_MT19937_32) return launch_jump_t<JMT32>(nullptr, gr, nitems, polys, s);
    if (variant == VMT_MT19937_64) return launch_jump_t<JMT64>(nullptr, gr, nitems, polys, s);
    return launch_jump_t<JSFMT>(nullptr, gr, nitems, polys, s);
}

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
