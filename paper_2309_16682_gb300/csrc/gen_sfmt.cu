// gen_sfmt.cu -- V-SFMT19937 generation kernel.
//
// SFMT19937 (Sec. 2.4) has a strictly serial chain: w_{k+N} depends on
// w_{k+N-1} (Sec. 2.6), so a single lane-state cannot be split along k.  The
// parallelism is across lanes and generators (the V-family's point, Sec. 3).
// Each lane-state is handled by four consecutive threads, thread j owning
// 32-bit sub-word j (sub-word 0 least significant) of all N = 156 elements in
// registers.  Per step of eq. (sfmt_step):
//   w_k <<< 8 needs sub-word j-1 of w_k          -> one shuffle
//   w_{k+N-2} >>> 8 needs sub-word j+1 of it     -> one shuffle
//   (w_{k+m} >> 11) & K and w_{k+N-1} << 18 are per sub-word.
// The block loop is fully unrolled so that every state index is static and
// the state never leaves registers.  Element (k, t) of generator g is written
// to S words 4(kM + t) + j: thread order (j, t, g) makes each warp store
// contiguous runs.
#include "vmt_device.cuh"

namespace vmt {
namespace dev {

constexpr int SF_N = 156, SF_M = 122;
constexpr int SF_THREADS = 128;

// emission of one 32-bit word (dtype chosen at run time, segments allowed)
__device__ __forceinline__ void sf_emit_generic(const GenArgs& a, long long g, long long f, uint32_t z,
                                                uint32_t partner, long long lo, long long hi, long long ebase)
{
    if (f < lo || f >= hi) return;
    const long long e = ebase + f - lo;
    int s = 0;
#pragma unroll
    for (int i = 1; i < VMT_MAXSEG; ++i)
        if (i < a.nseg && e >= a.seg[i].wbeg) s = i;
    const SegArg& sg = a.seg[s];
    const long long rel = e - sg.wbeg;
    const long long idx = g * sg.count;
    switch (sg.dtype) {
    case VMT_U32: __stcs(reinterpret_cast<uint32_t*>(sg.out) + idx + rel, z); break;
    case VMT_F32: __stcs(reinterpret_cast<float*>(sg.out) + idx + rel, f32_of_u32(z)); break;
    case VMT_U64:
        if ((rel & 1) == 0)
            __stcs(reinterpret_cast<unsigned long long*>(sg.out) + idx + rel / 2,
                   static_cast<unsigned long long>(z) | (static_cast<unsigned long long>(partner) << 32));
        break;
    case VMT_F64:
        if ((rel & 1) == 0) __stcs(reinterpret_cast<double*>(sg.out) + idx + rel / 2, f64_of_pair(z, partner));
        break;
    }
}

// PLAIN_U32: a single u32 segment; otherwise any segment list.
template <int M, bool PLAIN_U32>
__global__ void __launch_bounds__(SF_THREADS) gen_sfmt_kernel(GenArgs a)
{
    constexpr long long B = 4LL * SF_N * M;   // u32 words per block
    const long long gtid = static_cast<long long>(blockIdx.x) * SF_THREADS + threadIdx.x;
    const int j = static_cast<int>(threadIdx.x & 3);
    const long long ls = gtid >> 2;               // lane-state = g*M + t
    const long long g = ls / M;
    const int t = static_cast<int>(ls % M);
    const bool active = g < a.gens;
    const uint32_t K = kSfmtMask[j];
    const unsigned FULL = 0xFFFFFFFFu;

    uint32_t* gst = reinterpret_cast<uint32_t*>(a.states) + (active ? g : 0) * B + 4 * t + j;
    uint32_t w[SF_N];
#pragma unroll
    for (int k = 0; k < SF_N; ++k) w[k] = active ? gst[4LL * k * M] : 0u;

    const long long og = a.gen0 + g;
    long long e = 0;
    const long long p = a.pos;
    uint32_t* out_u32 = PLAIN_U32 ? reinterpret_cast<uint32_t*>(a.seg[0].out) + og * a.seg[0].count : nullptr;

    if (p < B && a.total > 0) {
        const long long hi = min(B, p + a.total);
#pragma unroll
        for (int k = 0; k < SF_N; ++k) {
            const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
            const uint32_t partner = __shfl_down_sync(FULL, w[k], 1, 4);
            if (!active) continue;
            if (PLAIN_U32) {
                if (f >= p && f < hi) __stcs(out_u32 + (f - p), w[k]);
            } else {
                sf_emit_generic(a, og, f, w[k], partner, p, hi, 0);
            }
        }
        e = hi - p;
    }
    while (e < a.total) {
        const long long hi = min(B, a.total - e);
#pragma unroll
        for (int k = 0; k < SF_N; ++k) {
            const uint32_t wa = w[k];
            const uint32_t wb = w[(k + SF_M) % SF_N];
            const uint32_t wc = w[(k + SF_N - 2) % SF_N];
            const uint32_t wd = w[(k + SF_N - 1) % SF_N];
            uint32_t am1 = __shfl_up_sync(FULL, wa, 1, 4);
            uint32_t cp1 = __shfl_down_sync(FULL, wc, 1, 4);
            if (j == 0) am1 = 0u;
            if (j == 3) cp1 = 0u;
            const uint32_t nw = wa ^ __funnelshift_l(am1, wa, 8) ^ ((wb >> 11) & K) ^ __funnelshift_r(wc, cp1, 8) ^
                                (wd << 18);
            w[k] = nw;
            const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
            if (PLAIN_U32) {
                if (active && f < hi) __stcs(out_u32 + e + f, nw);
            } else {
                const uint32_t partner = __shfl_down_sync(FULL, nw, 1, 4);
                if (active) sf_emit_generic(a, og, f, nw, partner, 0, hi, e);
            }
        }
        e += hi;
    }
    if (active) {
#pragma unroll
        for (int k = 0; k < SF_N; ++k) gst[4LL * k * M] = w[k];
    }
}

template <int M>
static cudaError_t launch_sfmt_m(const GenArgs& a, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    const long long threads = a.gens * M * 4;
    const long long grid = (threads + SF_THREADS - 1) / SF_THREADS;
    const bool plain = a.nseg == 1 && a.seg[0].dtype == VMT_U32;
    if (plain)
        gen_sfmt_kernel<M, true><<<static_cast<unsigned>(grid), SF_THREADS, 0, st>>>(a);
    else
        gen_sfmt_kernel<M, false><<<static_cast<unsigned>(grid), SF_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dev

cudaError_t launch_generate_sfmt(int lanes, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    switch (lanes) {
    case 1: return launch_sfmt_m<1>(a, s);
    case 2: return launch_sfmt_m<2>(a, s);
    case 4: return launch_sfmt_m<4>(a, s);
    case 8: return launch_sfmt_m<8>(a, s);
    case 16: return launch_sfmt_m<16>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace vmt
