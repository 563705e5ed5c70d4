// gen_mtc.cuh -- chain form of the V-MT19937-32 / V-MT19937-64 generation kernel.
//
// The recurrence eq. (step) in the modulo-free form eq. (stepnomod) makes a
// block of n new words per lane in three sub-loops: rows [0, n-m) read the old
// x_{k+m}; the later rows read the new word x'_{k-(n-m)} instead.  Cutting the
// block every n-m rows gives phases whose rows are independent (MT19937-32:
// 227/227/170, MT19937-64: 156/156).  The phase form (gen_mt.cu) hands every
// phase to all threads of the CTA and separates the phases by barriers.
//
// Here one thread owns a chain: rows j, j+(n-m) and j+2(n-m) of one vector
// column.  The new word a later row of the chain reads was made one step
// earlier by the same thread and is still in a register, so the rows of a
// block need no barrier among themselves; the only barrier of a block is the
// one before the two copies of X-hat swap.  The last row, k = n-1, also reads
// the new word 0 of its column (x_{k+1} = x'_0), which its thread recomputes
// from the old block with one more twist.
//
// Lanes never interact (Sec. 3: each lane is an independent copy of the base
// generator), so a CTA may own a group of L of the generator's M lanes: H =
// M/L CTAs share a generator without any exchange.  Each CTA keeps the
// n x L slice of X-hat (two copies) in shared memory; L words of a row are
// at least one 32-byte sector, so the output stays whole-sector stores and
// the interleaved order S[kM+t] (eq. combseq) is kept: lane t of row k goes to
// block word k*M + t.  Smaller slices let more CTAs share an SM.
//
// The state slice moves in with 16-byte asynchronous copies (cp.async) into
// the idle copy while the finished one is written back, and out with plain
// 16-byte stores.
#pragma once
#include "bulk.cuh"
#include "gen_mt.cuh"

namespace vmt {
namespace dev {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Geometry of one chain-form configuration: generator G, M lanes, L lanes per
// CTA, VW words per vector, T threads.
template <class G, int M, int L, int VW, int T>
struct ChainGeo {
    using W = typename G::W;
    static constexpr int N = G::N, MM = G::MM, NM = N - MM;
    static constexpr int H = M / L;          // CTAs per generator
    static constexpr int RV = L / VW;        // vectors per row of the slice
    static constexpr int NCH = NM * RV;      // chains
    static constexpr int CPT = (NCH + T - 1) / T;
    static constexpr int SLICE = N * L;      // words of one copy
    static constexpr int B = N * M;          // words of one generator block
    static constexpr int CPR = L * static_cast<int>(sizeof(W)) / 16;   // 16-byte chunks per row slice
    static constexpr int CHUNKS = N * CPR;
    static constexpr int SMEM = 2 * SLICE * static_cast<int>(sizeof(W));
    static_assert(M % L == 0 && L % VW == 0, "lane groups of whole vectors");
    static_assert(2 * NM <= N && N <= 3 * NM, "two or three phases");
    static_assert(CPR >= 1, "a row slice is at least 16 bytes");
};

// emit one tempered vector of the block at block word f0 (whole vectors
// inside [0, hi) and an aligned plan take the typed store)
template <class P, typename W, int VW>
__device__ __forceinline__ void chain_emit(const TypedPlan& plan, const Emitter& em, int f0, const W (&z)[VW], int hi,
                                           long long e, bool check)
{
    emit_p<P, W, VW>(plan, em, f0, z, 0, hi, e, true, check);
}

// One block of n new words for the CTA's slice: every chain of the thread,
// phase 1, 2 and (MT19937-32) 3 rows in order.
template <class G, int M, int L, int VW, int T, class P>
__device__ __forceinline__ void chain_block(const typename G::W* __restrict__ cur, typename G::W* __restrict__ nxt,
                                            const TypedPlan& plan, const Emitter& em, int fbase, int hi, long long e,
                                            bool check)
{
    using Geo = ChainGeo<G, M, L, VW, T>;
    using W = typename G::W;
    constexpr int N = Geo::N, MM = Geo::MM, NM = Geo::NM, RV = Geo::RV;
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < Geo::CPT; ++i) {
        const int c = tid + i * T;
        if ((i + 1) * T > Geo::NCH && c >= Geo::NCH) break;   // only the last round is partial
        const int j = c / RV;
        const int col = (c % RV) * VW;
        W xa[VW], xb[VW], xc[VW], nw[VW], z[VW];
        // phase 1: row j from the old x_j, x_{j+1}, x_{j+m}
        ldv<W, VW>(cur + j * L + col, xa);
        ldv<W, VW>(cur + (j + 1) * L + col, xb);
        ldv<W, VW>(cur + (j + MM) * L + col, xc);
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            nw[u] = G::twist(xa[u], xb[u], xc[u]);
            z[u] = G::temper(nw[u], em.a.k);
        }
        stv<W, VW>(nxt + j * L + col, nw);
        chain_emit<P, W, VW>(plan, em, j * M + fbase + col, z, hi, e, check);
        // phases 2 and 3: row k from the old x_k, x_{k+1} and the new x'_{k-(n-m)}
#pragma unroll
        for (int ph = 1; ph < 3; ++ph) {
            const int k = j + ph * NM;
            if (ph == 2 && (2 * NM >= N || k >= N)) break;
            ldv<W, VW>(cur + k * L + col, xa);
            if (k + 1 < N) {
                ldv<W, VW>(cur + (k + 1) * L + col, xb);
            } else {
                // x_{k+1} of the last row is the new word 0 of this column
                W a0[VW], a1[VW], am[VW];
                ldv<W, VW>(cur + col, a0);
                ldv<W, VW>(cur + L + col, a1);
                ldv<W, VW>(cur + MM * L + col, am);
#pragma unroll
                for (int u = 0; u < VW; ++u) xb[u] = G::twist(a0[u], a1[u], am[u]);
            }
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                nw[u] = G::twist(xa[u], xb[u], nw[u]);
                z[u] = G::temper(nw[u], em.a.k);
            }
            stv<W, VW>(nxt + k * L + col, nw);
            chain_emit<P, W, VW>(plan, em, k * M + fbase + col, z, hi, e, check);
        }
    }
}

template <class G, int M, int L, int VW, int T, int MINB, class P, bool UNITS>
__global__ void __launch_bounds__(T, MINB) gen_mtc_kernel(GenArgs a)
{
    using Geo = ChainGeo<G, M, L, VW, T>;
    using W = typename G::W;
    constexpr int N = Geo::N, H = Geo::H, RV = Geo::RV, B = Geo::B;
    static_assert(!UNITS || H == 1, "unit launches keep one CTA per generator");
    static_assert(!P::generic, "typed output policies only");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    W* const buf = reinterpret_cast<W*>(smem_raw);
    __shared__ long long s_next;
    const int tid = threadIdx.x;
    const long long items = UNITS ? a.gens : a.gens * H;

    auto state_of = [&](long long gi) -> W* {
        if constexpr (UNITS) return reinterpret_cast<W*>(a.units[gi].state);
        else return reinterpret_cast<W*>(a.states) + gi * static_cast<long long>(B);
    };
    // the 16-byte chunks of item u's slice: row r, piece p of the row
    auto load_slice = [&](W* dst, long long u) {
        const long long gi = UNITS ? u : u / H;
        const int h = UNITS ? 0 : static_cast<int>(u % H);
        const char* src = reinterpret_cast<const char*>(state_of(gi)) + h * L * sizeof(W);
        for (int ch = tid; ch < Geo::CHUNKS; ch += T) {
            const int r = ch / Geo::CPR, pc = ch % Geo::CPR;
            cp_async16(reinterpret_cast<char*>(dst) + r * L * sizeof(W) + pc * 16,
                       src + static_cast<long long>(r) * M * sizeof(W) + pc * 16);
        }
        cp_async_commit();
    };
    auto store_slice = [&](const W* s, long long u) {
        const long long gi = UNITS ? u : u / H;
        const int h = UNITS ? 0 : static_cast<int>(u % H);
        char* dst = reinterpret_cast<char*>(state_of(gi)) + h * L * sizeof(W);
        for (int ch = tid; ch < Geo::CHUNKS; ch += T) {
            const int r = ch / Geo::CPR, pc = ch % Geo::CPR;
            const uint4 v = *reinterpret_cast<const uint4*>(reinterpret_cast<const char*>(s) + r * L * sizeof(W) + pc * 16);
            *reinterpret_cast<uint4*>(dst + static_cast<long long>(r) * M * sizeof(W) + pc * 16) = v;
        }
    };
    const bool counter = UNITS && a.work_counter != nullptr;
    long long u;
    if (counter) {
        if (tid == 0) s_next = static_cast<long long>(atomicAdd(a.work_counter, 1));
        __syncthreads();
        u = s_next;
    } else {
        u = blockIdx.x;
    }
    int cb = 0;
    if (u < items) load_slice(buf, u);
    while (u < items) {
        cp_async_wait_all();
        __syncthreads();   // the slice is visible to all; the previous write-back has read its copy
        W* cur = buf + cb * Geo::SLICE;
        W* nxt = buf + (cb ^ 1) * Geo::SLICE;
        const long long gi = UNITS ? u : u / H;
        const int fbase = UNITS ? 0 : static_cast<int>(u % H) * L;   // first lane of the group
        const UnitDesc* ud = UNITS ? &a.units[gi] : nullptr;
        const Emitter em{a, a.gen0 + gi, UNITS ? ud->out : nullptr};
        int* posp = UNITS ? ud->pos : a.pos_dev + gi;
        const long long total = UNITS ? ud->total : a.total;
        const int p = UNITS ? *posp : a.pos;
        int final_pos = p;
        long long e = 0;
        TypedPlan plan;
        if (p < B && total > 0) {
            // rest of the current block: block word f is call word f - p
            const int hi = static_cast<int>(min(static_cast<long long>(B), p + total));
            plan.template make<P, W, VW>(a, em, -static_cast<long long>(p));
            for (int v = tid; v < N * RV; v += T) {
                const int k = v / RV, col = (v % RV) * VW;
                const int f0 = k * M + fbase + col;
                const bool act = f0 + VW > p && f0 < hi;
                W z[VW];
                if (act) {
                    W w[VW];
                    ldv<W, VW>(cur + k * L + col, w);
#pragma unroll
                    for (int q = 0; q < VW; ++q) z[q] = G::temper(w[q], a.k);
                } else {
#pragma unroll
                    for (int q = 0; q < VW; ++q) z[q] = W(0);
                }
                emit_p<P, W, VW>(plan, em, f0, z, p, hi, -static_cast<long long>(p), act, true);
            }
            e = hi - p;
            final_pos = hi;
        }
        while (e < total) {
            const int hi = static_cast<int>(min(static_cast<long long>(B), total - e));   // block words [0, hi) emitted
            plan.template make<P, W, VW>(a, em, e);
            chain_block<G, M, L, VW, T, P>(cur, nxt, plan, em, fbase, hi, e, hi < B);
            __syncthreads();
            W* t = cur;
            cur = nxt;
            nxt = t;
            cb ^= 1;
            e += hi;
            final_pos = hi;
        }
        // the next item's slice into the idle copy while this one is written back
        long long un;
        if (counter) {
            if (tid == 0) s_next = static_cast<long long>(atomicAdd(a.work_counter, 1));
            __syncthreads();
            un = s_next;
        } else {
            un = u + gridDim.x;
        }
        if (un < items) load_slice(nxt, un);
        store_slice(cur, u);
        if (tid == 0 && fbase == 0) *posp = final_pos;   // every group of a generator ends at the same position
        cb ^= 1;
        u = un;
    }
    cp_async_wait_all();
}

// resident CTAs per SM of one instantiation (occupancy query, cached)
template <class K>
static int resident_ctas(K kernel, int threads, int smem)
{
    static int cached = 0;
    if (!cached) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
        cached = n;
    }
    return cached;
}

template <class G, int M, int L, int VW, int T, int MINB, class P, bool UNITS>
static cudaError_t launch_mtc_pu(const GenArgs& a, cudaStream_t st)
{
    using Geo = ChainGeo<G, M, L, VW, T>;
    auto kern = gen_mtc_kernel<G, M, L, VW, T, MINB, P, UNITS>;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Geo::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const long long items = UNITS ? a.gens : a.gens * Geo::H;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long persistent = static_cast<long long>(sms) * resident_ctas(kern, T, Geo::SMEM);
    // unit launches may ask for one CTA per unit (each then takes one unit)
    const long long cap = (UNITS && a.cta_per_unit) ? items : persistent;
    const long long grid = items < cap ? items : cap;
    kern<<<static_cast<unsigned>(grid), T, Geo::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <class G, int M, int L, int VW, int T, int MINB, class P>
static cudaError_t launch_mtc_p(const GenArgs& a, cudaStream_t st)
{
    if (a.units) {
        if constexpr (L == M) return launch_mtc_pu<G, M, L, VW, T, MINB, P, true>(a, st);
        return cudaErrorNotSupported;
    }
    return launch_mtc_pu<G, M, L, VW, T, MINB, P, false>(a, st);
}

// typed policies only: the other output patterns are not supported here
template <class G, int M, int L, int VW, int T, int MINB>
static cudaError_t launch_mtc(const GenArgs& a, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    const int d0 = a.seg[0].dtype, d1 = a.nseg > 1 ? a.seg[1].dtype : -1;
    if constexpr (sizeof(typename G::W) == 4) {
        if (a.nseg == 1 && d0 == VMT_U32) return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_U32, -1>>(a, st);
        if (a.nseg == 1 && d0 == VMT_F32) return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_F32, -1>>(a, st);
        if (a.nseg == 1 && d0 == VMT_F64) return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_F64, -1>>(a, st);
        if (a.nseg == 2 && d0 == VMT_U32 && d1 == VMT_F32)
            return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_U32, VMT_F32>>(a, st);
    } else {
        if (a.nseg == 1 && d0 == VMT_U64) return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_U64, -1>>(a, st);
        if (a.nseg == 1 && d0 == VMT_F64) return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_F64, -1>>(a, st);
        if (a.nseg == 2 && d0 == VMT_U64 && d1 == VMT_F64)
            return launch_mtc_p<G, M, L, VW, T, MINB, Pol<VMT_U64, VMT_F64>>(a, st);
    }
    return cudaErrorNotSupported;
}

}  // namespace dev
}  // namespace vmt
