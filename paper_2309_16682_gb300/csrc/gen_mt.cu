// gen_mt.cu -- V-MT19937-32 and V-MT19937-64 generation kernels.
//
// One CTA owns one V-generator: its combined state X-hat (Sec. 3), n rows of
// M lane words with row k holding word k of every lane, is staged in shared
// memory in exactly the paper's interleaved order.  With that layout the
// output sequence S (eq. combseq) of a block is the tempered state read in
// memory order, so the interleave costs nothing and every thread writes one
// contiguous 16-byte vector.
//
// A new block of n words per lane is produced by the recurrence eq. (step)
// in the modulo-free form eq. (stepnomod): rows [0, n-m) read x_{k+m} of the
// old block, later rows read the new word x'_{k-(n-m)} written (n-m) rows
// earlier.  Cutting the block every n-m rows therefore gives phases whose rows
// are independent (MT19937-32: 227/227/170 rows, MT19937-64: 156/156 rows).
// Within a phase, row k also reads the old x_{k+1} that row k+1 overwrites, so
// each phase loads all operands, synchronises, then writes.
#include "vmt_device.cuh"

namespace vmt {
namespace dev {

template <typename W, int VW> struct VecOf;
template <> struct VecOf<uint32_t, 4> { using T = uint4; };
template <> struct VecOf<uint32_t, 2> { using T = uint2; };
template <> struct VecOf<uint32_t, 1> { using T = uint32_t; };
template <> struct VecOf<unsigned long long, 2> { using T = ulonglong2; };
template <> struct VecOf<unsigned long long, 1> { using T = unsigned long long; };

template <typename W, int VW>
__device__ __forceinline__ void ldv(const W* p, W (&w)[VW])
{
    using T = typename VecOf<W, VW>::T;
    const T t = *reinterpret_cast<const T*>(p);
    memcpy(w, &t, sizeof(T));
}

template <typename W, int VW>
__device__ __forceinline__ void stv(W* p, const W (&w)[VW])
{
    using T = typename VecOf<W, VW>::T;
    T t;
    memcpy(&t, w, sizeof(T));
    *reinterpret_cast<T*>(p) = t;
}

template <int VW>
__device__ __forceinline__ void emit_words(const Emitter& em, long long f0, const uint32_t (&z)[VW], long long lo,
                                           long long hi, long long ebase)
{
    em.emit32<VW>(f0, z, lo, hi, ebase);
}

template <int VW>
__device__ __forceinline__ void emit_words(const Emitter& em, long long f0, const unsigned long long (&z)[VW],
                                           long long lo, long long hi, long long ebase)
{
    em.emit64<VW>(f0, z, lo, hi, ebase);
}

template <class G, int M, int VW, int T>
__global__ void __launch_bounds__(T) gen_mt_kernel(GenArgs a)
{
    using W = typename G::W;
    constexpr int N = G::N, MM = G::MM, NM = N - MM;
    constexpr int B = N * M;        // words per block
    constexpr int RV = M / VW;      // vectors per row
    constexpr int NV = B / VW;      // vectors per block
    constexpr int ITEMS = (NM * RV + T - 1) / T;
    __shared__ __align__(16) W s[B];

    for (long long gi = blockIdx.x; gi < a.gens; gi += gridDim.x) {
        W* gst = reinterpret_cast<W*>(a.states) + gi * static_cast<long long>(B);
        for (int v = threadIdx.x; v < NV; v += T) {
            W w[VW];
            ldv<W, VW>(gst + v * VW, w);
            stv<W, VW>(s + v * VW, w);
        }
        __syncthreads();
        const Emitter em{a, a.gen0 + gi};
        long long e = 0;
        const long long p = a.pos;
        if (p < B && a.total > 0) {
            // rest of the current block
            const long long hi = min(static_cast<long long>(B), p + a.total);
            for (long long v = p / VW + threadIdx.x; v * VW < hi; v += T) {
                W w[VW], z[VW];
                ldv<W, VW>(s + v * VW, w);
#pragma unroll
                for (int u = 0; u < VW; ++u) z[u] = G::temper(w[u]);
                emit_words<VW>(em, v * VW, z, p, hi, 0);
            }
            e = hi - p;
        }
        while (e < a.total) {
            const long long hi = min(static_cast<long long>(B), a.total - e);
#pragma unroll 1
            for (int k0 = 0; k0 < N; k0 += NM) {
                const int k1 = min(k0 + NM, N);
                const int v0 = k0 * RV, v1 = k1 * RV;
                W xa[ITEMS][VW], xb[ITEMS][VW], xc[ITEMS][VW];
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const int v = v0 + static_cast<int>(threadIdx.x) + i * T;
                    if (v < v1) {
                        ldv<W, VW>(s + v * VW, xa[i]);
                        int vb = v + RV;
                        if (vb >= NV) vb -= NV;   // x_{n} of the last row is the new x_0
                        ldv<W, VW>(s + vb * VW, xb[i]);
                        const int vc = (k0 == 0) ? v + MM * RV : v - NM * RV;
                        ldv<W, VW>(s + vc * VW, xc[i]);
                    }
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const int v = v0 + static_cast<int>(threadIdx.x) + i * T;
                    if (v < v1) {
                        W nw[VW], z[VW];
#pragma unroll
                        for (int u = 0; u < VW; ++u) {
                            nw[u] = G::twist(xa[i][u], xb[i][u], xc[i][u]);
                            z[u] = G::temper(nw[u]);
                        }
                        stv<W, VW>(s + v * VW, nw);
                        emit_words<VW>(em, static_cast<long long>(v) * VW, z, 0, hi, e);
                    }
                }
                __syncthreads();
            }
            e += hi;
        }
        for (int v = threadIdx.x; v < NV; v += T) {
            W w[VW];
            ldv<W, VW>(s + v * VW, w);
            stv<W, VW>(gst + v * VW, w);
        }
        __syncthreads();
    }
}

template <class G, int M, int VW, int T>
static cudaError_t launch_mt(const GenArgs& a, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    const long long grid = a.gens < (1LL << 30) ? a.gens : (1LL << 30);
    gen_mt_kernel<G, M, VW, T><<<static_cast<unsigned>(grid), T, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace dev

cudaError_t launch_generate_mt(int variant, int lanes, const GenArgs& a, cudaStream_t s)
{
    using namespace dev;
    if (variant == VMT_MT19937_32) {
        switch (lanes) {
        case 1: return launch_mt<MT32, 1, 1, 256>(a, s);
        case 2: return launch_mt<MT32, 2, 2, 256>(a, s);
        case 4: return launch_mt<MT32, 4, 4, 256>(a, s);
        case 8: return launch_mt<MT32, 8, 4, 256>(a, s);
        case 16: return launch_mt<MT32, 16, 4, 512>(a, s);
        }
    } else if (variant == VMT_MT19937_64) {
        switch (lanes) {
        case 1: return launch_mt<MT64, 1, 1, 256>(a, s);
        case 2: return launch_mt<MT64, 2, 2, 256>(a, s);
        case 4: return launch_mt<MT64, 4, 2, 256>(a, s);
        case 8: return launch_mt<MT64, 8, 2, 256>(a, s);
        case 16: return launch_mt<MT64, 16, 2, 512>(a, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace vmt
