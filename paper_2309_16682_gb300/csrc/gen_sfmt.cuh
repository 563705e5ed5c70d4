// gen_sfmt.cuh -- V-SFMT19937 generation kernel (instantiated per lane count in
// gen_sfmt_m*.cu so that the heavy unrolled instances compile in parallel).
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
#pragma once
#include "vmt_device.cuh"

namespace vmt {
namespace dev {

constexpr int SF_N = 156, SF_M = 122;
constexpr int SF_THREADS = 128;

// emission of one 32-bit word (dtype chosen at run time, segments allowed)
__device__ __forceinline__ void sf_emit_generic(const Emitter& em, long long f, uint32_t z, uint32_t partner,
                                                long long lo, long long hi, long long ebase)
{
    if (f < lo || f >= hi) return;
    const long long e = ebase + f - lo;
    const int s = em.seg_of(e);
    const SegArg& sg = em.a.seg[s];
    const long long rel = e - sg.wbeg;
    char* base = em.elem0(s);
    switch (sg.dtype) {
    case VMT_U32: __stcs(reinterpret_cast<uint32_t*>(base) + rel, z); break;
    case VMT_F32: __stcs(reinterpret_cast<float*>(base) + rel, f32_of_u32(z)); break;
    case VMT_U64:
        if ((rel & 1) == 0)
            __stcs(reinterpret_cast<unsigned long long*>(base) + rel / 2,
                   static_cast<unsigned long long>(z) | (static_cast<unsigned long long>(partner) << 32));
        break;
    case VMT_F64:
        if ((rel & 1) == 0) __stcs(reinterpret_cast<double*>(base) + rel / 2, f64_of_pair(z, partner));
        break;
    }
}

// PLAIN_U32: a single u32 segment; otherwise any segment list.
// RAGGED: the lane-states of a warp may start at different positions or need
// different lengths; a lane-state that is done keeps its registers unchanged
// while the others of its warp continue.
template <int M, bool PLAIN_U32, bool RAGGED>
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

    // non-ragged launches: one position and one length for every lane-state,
    // taken from the kernel parameters (uniform values)
    const UnitDesc* ud = (RAGGED && a.units && active) ? &a.units[g] : nullptr;
    uint32_t* gbase = ud ? reinterpret_cast<uint32_t*>(ud->state) : reinterpret_cast<uint32_t*>(a.states) + (active ? g : 0) * B;
    uint32_t* gst = gbase + 4 * t + j;
    int* posp = ud ? ud->pos : a.pos_dev + (active ? g : 0);
    const long long total = RAGGED ? (active ? (ud ? ud->total : a.total) : 0) : a.total;
    const long long p = RAGGED ? (active ? *posp : B) : a.pos;
    const Emitter em{a, a.gen0 + g, ud ? ud->out : nullptr};

    uint32_t w[SF_N];
#pragma unroll
    for (int k = 0; k < SF_N; ++k) w[k] = active ? gst[4LL * k * M] : 0u;

    long long e = 0;
    long long final_pos = p;
    uint32_t* out_u32 = (PLAIN_U32 && active) ? reinterpret_cast<uint32_t*>(em.elem0(0)) : nullptr;

    if constexpr (!RAGGED) {
        // one position and one length for the whole launch: uniform loops
        if (p < B && total > 0) {
            const long long hi = min(B, p + total);
#pragma unroll
            for (int k = 0; k < SF_N; ++k) {
                const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
                const uint32_t partner = __shfl_down_sync(FULL, w[k], 1, 4);
                if (!active) continue;
                if (PLAIN_U32) {
                    if (f >= p && f < hi) __stcs(out_u32 + (f - p), w[k]);
                } else {
                    sf_emit_generic(em, f, w[k], partner, p, hi, 0);
                }
            }
            e = hi - p;
            final_pos = hi;
        }
        while (e < total) {
            const long long hi = min(B, total - e);
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
                const uint32_t nw = wa ^ __funnelshift_l(am1, wa, 8) ^ ((wb >> 11) & K) ^
                                    __funnelshift_r(wc, cp1, 8) ^ (wd << 18);
                w[k] = nw;
                const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
                if (PLAIN_U32) {
                    if (active && f < hi) __stcs(out_u32 + e + f, nw);
                } else {
                    const uint32_t partner = __shfl_down_sync(FULL, nw, 1, 4);
                    if (active) sf_emit_generic(em, f, nw, partner, 0, hi, e);
                }
            }
            e += hi;
            final_pos = hi;
        }
    } else {
        // lane-states of a warp differ in position or length
        if (__any_sync(FULL, active && p < B && total > 0)) {
            const bool mine = active && p < B && total > 0;
            const long long hi = mine ? min(B, p + total) : 0;
#pragma unroll
            for (int k = 0; k < SF_N; ++k) {
                const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
                const uint32_t partner = __shfl_down_sync(FULL, w[k], 1, 4);
                if (!mine) continue;
                if (PLAIN_U32) {
                    if (f >= p && f < hi) __stcs(out_u32 + (f - p), w[k]);
                } else {
                    sf_emit_generic(em, f, w[k], partner, p, hi, 0);
                }
            }
            if (mine) {
                e = hi - p;
                final_pos = hi;
            }
        }
        while (__any_sync(FULL, active && e < total)) {
            const bool live = active && e < total;
            const long long hi = live ? min(B, total - e) : 0;
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
                const uint32_t nw = wa ^ __funnelshift_l(am1, wa, 8) ^ ((wb >> 11) & K) ^
                                    __funnelshift_r(wc, cp1, 8) ^ (wd << 18);
                w[k] = live ? nw : wa;   // a finished lane-state keeps its state
                const long long f = 4LL * (static_cast<long long>(k) * M + t) + j;
                if (PLAIN_U32) {
                    if (live && f < hi) __stcs(out_u32 + e + f, nw);
                } else {
                    const uint32_t partner = __shfl_down_sync(FULL, nw, 1, 4);
                    if (live) sf_emit_generic(em, f, nw, partner, 0, hi, e);
                }
            }
            if (live) {
                e += hi;
                final_pos = hi;
            }
        }
    }
    if (active) {
#pragma unroll
        for (int k = 0; k < SF_N; ++k) gst[4LL * k * M] = w[k];
        if (t == 0 && j == 0) *posp = static_cast<int>(final_pos);
    }
}

template <int M>
cudaError_t launch_sfmt_m(const GenArgs& a, bool ragged, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    const long long threads = a.gens * M * 4;
    const long long grid = (threads + SF_THREADS - 1) / SF_THREADS;
    const bool plain = a.nseg == 1 && a.seg[0].dtype == VMT_U32;
    const unsigned gr = static_cast<unsigned>(grid);
    if (plain && !ragged) gen_sfmt_kernel<M, true, false><<<gr, SF_THREADS, 0, st>>>(a);
    else if (plain) gen_sfmt_kernel<M, true, true><<<gr, SF_THREADS, 0, st>>>(a);
    else if (!ragged) gen_sfmt_kernel<M, false, false><<<gr, SF_THREADS, 0, st>>>(a);
    else gen_sfmt_kernel<M, false, true><<<gr, SF_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dev
}  // namespace vmt
