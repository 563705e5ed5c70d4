// gen_mt_kernel.cuh -- V-MT19937-32 and V-MT19937-64 generation kernels
// (instantiated per variant in gen_mt32.cu and gen_mt64.cu, dispatched from
// gen_mt.cu).
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
// The two copies of X-hat (old block read, new block written) let a phase
// load and store without a barrier in between.
//
// Any cut works as long as no item (one vector of M / VW lanes of a row)
// shares a pass with the item (n-m) rows before it; twist_block picks the cut
// (MT19937-32 with 16 lanes and 512 threads: 2496 items in five passes of one
// item per thread instead of three phases of up to two items each).
//
// In place (template flag IP): one copy of X-hat, half the shared memory, so
// that five 256-thread CTAs share an SM.  Of an item's operands only the old
// x_{k+1} may be overwritten by another thread in the same pass; each thread
// loads those of its next pass before the barrier that starts it (see
// preload_next and early_first_preload; tests/test_pass_schedule_cpu.py
// replays the schedule of every compiled configuration).
#pragma once
#include "bulk.cuh"
#include "gen_mt.cuh"
#include "pass_cut.hpp"

namespace vmt {
namespace dev {

// One item of a pass over vectors [V0, V1) of the block: vector v of the new
// block from the old block `cur` and the rows of `nxt` finished by earlier
// passes; the new words are written to nxt and returned in nw.  In place
// (IP: cur == nxt, one copy of X-hat) the old x_{k+1}, which another thread
// overwrites in this pass, was loaded into pb before the previous barrier.
template <class G, int M, int VW, int V0, int V1, bool IP>
__device__ __forceinline__ void twist_vec(const typename G::W* cur, typename G::W* nxt, int v,
                                          typename G::W (&nw)[VW], const ShiftK& k, const typename G::W (&pb)[VW])
{
    using W = typename G::W;
    constexpr int N = G::N, MM = G::MM, NM = N - MM;
    constexpr int RV = M / VW, NV = N * RV, DV = NM * RV;
    W xa[VW], xb[VW], xc[VW];
    ldv<W, VW>(cur + v * VW, xa);
    if (V1 <= NV - RV || v + RV < NV) {                                       // old x_{k+1}
        if constexpr (IP) {
#pragma unroll
            for (int u = 0; u < VW; ++u) xb[u] = pb[u];
        } else {
            ldv<W, VW>(cur + (v + RV) * VW, xb);
        }
    } else {
        ldv<W, VW>(nxt + (v + RV - NV) * VW, xb);                           // new x_0 for the last row
    }
    if (V1 <= DV || (V0 < DV && v < DV)) ldv<W, VW>(cur + (v + MM * RV) * VW, xc);   // old x_{k+m}
    else ldv<W, VW>(nxt + (v - DV) * VW, xc);                                      // new x_{k-(n-m)}
#pragma unroll
    for (int u = 0; u < VW; ++u) nw[u] = G::twist(xa[u], xb[u], xc[u], k);
    stv<W, VW>(nxt + v * VW, nw);
}

template <class G, int M, int VW, int V0, int V1, bool IP>
__device__ __forceinline__ void twist_item(const typename G::W* cur, typename G::W* nxt, int v,
                                           typename G::W (&z)[VW], const ShiftK& k, const typename G::W (&pb)[VW])
{
    typename G::W nw[VW];
    twist_vec<G, M, VW, V0, V1, IP>(cur, nxt, v, nw, k, pb);
#pragma unroll
    for (int u = 0; u < VW; ++u) z[u] = G::temper(nw[u], k);
}

// One pass of the block twist: vectors [V0, V1), thread tid taking V0 + tid,
// V0 + tid + T, ...  When the whole pass is emitted into one statically typed
// segment (the common case) the items run without any per-vector check;
// otherwise every vector is routed by emit_p.
template <class G, int M, int VW, int T, class P, int V0, int V1, bool IP, int IMAX>
__device__ __forceinline__ void twist_pass(const typename G::W* cur, typename G::W* nxt,
                                           const typename PlanOf<P>::type& plan, const Emitter& em, int hi,
                                           long long e, bool check, const typename G::W (&pre)[IMAX][VW])
{
    using W = typename G::W;
    constexpr int ITEMS = (V1 - V0 + T - 1) / T;
    static_assert(ITEMS <= IMAX, "preload slots");
    const int tid = threadIdx.x;
    if constexpr (!P::generic) {
        const bool inside = !check || V1 * VW <= hi;   // every vector of the pass is emitted
        if (inside && plan.ok && (P::nseg == 1 || plan.b1 >= V1 * VW || plan.b1 <= V0 * VW)) {
            const bool second = P::nseg == 2 && plan.b1 <= V0 * VW;
            const long long base = second ? plan.base1 : plan.base0;
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int v = V0 + tid + i * T;
                if (((i + 1) * T <= V1 - V0) || v < V1) {
                    W z[VW];
                    twist_item<G, M, VW, V0, V1, IP>(cur, nxt, v, z, em.a.k, pre[i]);
                    if (P::nseg == 2 && second) store_typed<(P::nseg == 2 ? P::DT1 : P::DT0), W, VW>(base, v * VW, z);
                    else store_typed<P::DT0, W, VW>(base, v * VW, z);
                }
            }
            return;
        }
        if (plan.ok) {
            // a pass that holds the end of the call's output or the segment
            // boundary: a whole vector inside [0, hi) takes the typed store of
            // its segment (the boundary falls between vectors), the vector
            // that straddles hi the word path, vectors at or beyond hi only
            // advance the state
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const int v = V0 + tid + i * T;
                if (((i + 1) * T <= V1 - V0) || v < V1) {
                    W nw[VW], z[VW];
                    twist_vec<G, M, VW, V0, V1, IP>(cur, nxt, v, nw, em.a.k, pre[i]);
                    const int f0 = v * VW;
                    if (f0 >= hi) continue;   // past the call's output: the state only
#pragma unroll
                    for (int u = 0; u < VW; ++u) z[u] = G::temper(nw[u], em.a.k);
                    if (f0 + VW <= hi) {
                        if (P::nseg == 2 && f0 >= plan.b1)
                            store_typed<(P::nseg == 2 ? P::DT1 : P::DT0), W, VW>(plan.base1, f0, z);
                        else
                            store_typed<P::DT0, W, VW>(plan.base0, f0, z);
                    } else if (f0 < hi) {
                        emit_words<VW>(em, f0, z, 0, hi, e);
                    }
                }
            }
            return;
        }
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int v = V0 + tid + i * T;
        const bool act = ((i + 1) * T <= V1 - V0) || v < V1;   // static for all but the last item
        W z[VW];
        if (act) twist_item<G, M, VW, V0, V1, IP>(cur, nxt, v, z, em.a.k, pre[i]);
        else {
#pragma unroll
            for (int u = 0; u < VW; ++u) z[u] = W(0);
        }
        emit_p<P, W, VW>(plan, em, v * VW, z, 0, hi, e, act, check);
    }
}

// In place: load the old x_{k+1} of the items of pass [A, B) (row k+1 of
// the same column, vector v + M / VW) into pre.  Those rows belong to that
// pass or the next one, so nobody writes them before pass [A, B) starts; the
// load must come before the barrier that starts it (another thread writes
// them in it).  The last row's x_{k+1} is the new x_0, read in its pass.
template <class G, int M, int VW, int T, int A, int B, int IMAX>
__device__ __forceinline__ void preload_next(const typename G::W* cur, typename G::W (&pre)[IMAX][VW])
{
    constexpr int RV = M / VW, NV = G::N * RV;
    constexpr int ITEMS = (B - A + T - 1) / T;
    static_assert(ITEMS <= IMAX, "preload slots");
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) {
        const int v = A + static_cast<int>(threadIdx.x) + i * T;
        if (v < B && v + RV < NV) ldv<typename G::W, VW>(cur + (v + RV) * VW, pre[i]);
    }
}

template <class G, int M, int VW, int T>
__host__ __device__ constexpr int block_step()
{
    return pass_step(G::N * (M / VW), (G::N - G::MM) * (M / VW), T);
}

template <class G, int M, int VW, int T>
__host__ __device__ constexpr bool early_first_preload()
{
    return vmt::early_first_preload(G::N * (M / VW), block_step<G, M, VW, T>(), M / VW);
}

// The passes from vector V0 on, each followed by a barrier.
template <class G, int M, int VW, int T, class P, bool IP, int V0, int IMAX>
__device__ __forceinline__ void twist_block(const typename G::W* cur, typename G::W* nxt,
                                            const typename PlanOf<P>::type& plan, const Emitter& em, int hi,
                                            long long e, bool check, typename G::W (&pre)[IMAX][VW])
{
    constexpr int N = G::N, NM = N - G::MM;
    constexpr int RV = M / VW, NV = N * RV, DV = NM * RV;
    constexpr int STEP = block_step<G, M, VW, T>();
    static_assert(STEP >= 1 && STEP <= DV, "a pass holds no dependent vectors");
    constexpr int V1 = V0 + STEP < NV ? V0 + STEP : NV;
    constexpr bool EARLY = early_first_preload<G, M, VW, T>();
    if constexpr (IP && V0 == 0 && !EARLY) {
        preload_next<G, M, VW, T, 0, V1, IMAX>(cur, pre);
        __syncthreads();
    }
    twist_pass<G, M, VW, T, P, V0, V1, IP, IMAX>(cur, nxt, plan, em, hi, e, check, pre);
    // in place: the next pass's operands, or after the last pass those of the
    // next block's first pass
    if constexpr (IP && V1 < NV) preload_next<G, M, VW, T, V1, (V1 + STEP < NV ? V1 + STEP : NV), IMAX>(cur, pre);
    if constexpr (IP && V1 == NV && EARLY) preload_next<G, M, VW, T, 0, STEP, IMAX>(cur, pre);
    __syncthreads();
    if constexpr (V1 < NV) twist_block<G, M, VW, T, P, IP, V1, IMAX>(cur, nxt, plan, em, hi, e, check, pre);
}

// set by a kernel whose bounded wait on a bulk copy gave up (one flag per
// translation unit that instantiates these kernels; see read_timeout_flag)
static __device__ int g_gen_timeout = 0;

// CTAs that fit on one SM: by threads (2048), by shared memory (two copies of
// X-hat per CTA out of 227 KiB) and by registers; the register budget of the
// launch bound follows from it.
template <class G, int M, int T, bool IP>
constexpr int mt_ctas_per_sm()
{
    constexpr int by_threads = 2048 / T;
    constexpr int copies = IP ? 1 : 2;
    constexpr int by_smem = (227 * 1024) / (copies * G::N * M * static_cast<int>(sizeof(typename G::W)) + 1024);
    constexpr int c = by_threads < by_smem ? by_threads : by_smem;
    // at least 48 registers a thread (fewer spill)
    constexpr int by_regs = 65536 / (T * 48);
    constexpr int r = c < by_regs ? c : by_regs;
    return r < 1 ? 1 : r;
}

template <class G, int M, int VW, int T, bool IP, class P, bool UNITS>
__global__ void __launch_bounds__(T, (mt_ctas_per_sm<G, M, T, IP>())) gen_mt_kernel(GenArgs a)
{
    using W = typename G::W;
    constexpr int N = G::N;
    constexpr int B = N * M;        // words per block
    constexpr uint32_t BYTES = static_cast<uint32_t>(B * sizeof(W));
    static_assert(N <= 3 * (N - G::MM), "at most three phases in the phase form");
    static_assert(BYTES % 16 == 0, "bulk copies move multiples of 16 bytes");
    // Two copies of X-hat: the old block is only read while the new one is
    // written, so a pass needs no barrier between its loads and its stores,
    // and the next generator's state is fetched into the idle copy while the
    // finished one is written back.  In place (IP): one copy, half the shared
    // memory (more CTAs per SM); each pass's x_{k+1} operands are loaded
    // before the barrier that starts it, and the next generator's state is
    // fetched once the write-back has read the copy.  A generator's state
    // arrives and leaves with one bulk copy each.
    extern __shared__ __align__(128) unsigned char smem_raw[];
    W* const buf0 = reinterpret_cast<W*>(smem_raw);
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x;
    using Plan = typename PlanOf<P>::type;

    __shared__ long long s_next;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    // Generators (lock-step) or units (ragged / batched launches) are taken
    // either in grid-stride order or, with a work counter, dynamically in the
    // order of the unit list (longest first).  Thread 0 fetches the next one
    // and starts the bulk copy of its state.
    long long my_next = blockIdx.x;   // grid-stride cursor (thread 0)
    auto take = [&]() -> long long {
        if (UNITS && a.work_counter) return static_cast<long long>(atomicAdd(a.work_counter, 1));
        const long long u = my_next;
        my_next += gridDim.x;
        return u;
    };
    auto state_of = [&](long long u) -> W* {
        if constexpr (UNITS) return reinterpret_cast<W*>(a.units[u].state);
        else return reinterpret_cast<W*>(a.states) + u * static_cast<long long>(B);
    };
    uint32_t parity = 0;
    int cb = 0;   // copy that holds the current state
    if (tid == 0) {
        const long long u = take();
        s_next = u;
        if (u < a.gens) {
            mbar_arrive_expect_tx(&bar, BYTES);
            bulk_load(buf0, state_of(u), BYTES, &bar);
        }
    }
    __syncthreads();
    long long gi = s_next;

    while (gi < a.gens) {
        W* gst = state_of(gi);
        const bool arrived = mbar_wait(&bar, parity);
        parity ^= 1u;
        if (__syncthreads_or(!arrived)) {
            if (tid == 0) {
                atomicExch(&g_gen_timeout, 1);
                (void)mbar_wait(&bar, parity ^ 1u);   // give the late copy one more bounded chance
                bulk_wait_all();
            }
            return;
        }
        W* cur = buf0 + cb * B;
        W* nxt = IP ? cur : buf0 + (cb ^ 1) * B;
        // lock-step launches take position and length from the kernel
        // parameters (uniform values); unit launches from the unit table
        const UnitDesc* ud = UNITS ? &a.units[gi] : nullptr;
        const Emitter em{a, a.gen0 + gi, UNITS ? ud->out : nullptr};
        int* posp = UNITS ? ud->pos : a.pos_dev + gi;
        const int total = static_cast<int>(UNITS ? ud->total : a.total);
        int e = 0;
        const int p = UNITS ? *posp : a.pos;
        int final_pos = p;
        Plan plan;
        if (p < B && total > 0) {
            // rest of the current block: block word f is call word f - p
            const int hi = min(B, p + total);
            plan.template make<P, W, VW>(a, em, -static_cast<long long>(p));
            bool done_head = false;
            if constexpr (!P::generic) {
                if (plan.ok) {
                    // whole vectors inside [p, hi) take the typed store of their
                    // segment, the ones that straddle p or hi the word path
                    for (int v = p / VW + tid; v * VW < hi; v += T) {
                        const int f0 = v * VW;
                        W w[VW], z[VW];
                        ldv<W, VW>(cur + f0, w);
#pragma unroll
                        for (int u = 0; u < VW; ++u) z[u] = G::temper(w[u], a.k);
                        if (f0 >= p && f0 + VW <= hi) {
                            if (P::nseg == 2 && f0 >= plan.b1)
                                store_typed<(P::nseg == 2 ? P::DT1 : P::DT0), W, VW>(plan.base1, f0, z);
                            else
                                store_typed<P::DT0, W, VW>(plan.base0, f0, z);
                        } else {
                            emit_words<VW>(em, f0, z, p, hi, 0);
                        }
                    }
                    done_head = true;
                }
            }
            if (!done_head) {
                for (int v0 = p / VW; v0 * VW < hi; v0 += T) {
                    const int v = v0 + tid;
                    W w[VW], z[VW];
                    const bool act = v * VW < hi;
                    if (act) ldv<W, VW>(cur + v * VW, w);
#pragma unroll
                    for (int u = 0; u < VW; ++u) z[u] = act ? G::temper(w[u], a.k) : W(0);
                    emit_p<P, W, VW>(plan, em, v * VW, z, p, hi, -static_cast<long long>(p), act, true);
                }
            }
            e = hi - p;
            final_pos = hi;
        }
        constexpr int IMAX = (block_step<G, M, VW, T>() + T - 1) / T;   // items per thread per pass
        W pre[IMAX][VW];
        if constexpr (IP) {
            // the first block's first-pass operands, then a barrier: the head
            // above still reads words that the block overwrites
            if (e < total) {
                if constexpr (early_first_preload<G, M, VW, T>())
                    preload_next<G, M, VW, T, 0, block_step<G, M, VW, T>(), IMAX>(cur, pre);
                __syncthreads();
            }
        }
        while (e < total) {
            const int hi = min(B, total - e);   // block words [0, hi) are emitted
            const bool check = hi < B;
            plan.template make<P, W, VW>(a, em, e);
            twist_block<G, M, VW, T, P, IP, 0, IMAX>(cur, nxt, plan, em, hi, e, check, pre);
            if constexpr (!IP) {
                W* t = cur;
                cur = nxt;
                nxt = t;
                cb ^= 1;
            }
            e += hi;
            final_pos = hi;
        }
        // write the state back and fetch the next generator's into the idle
        // copy (in place: into the same copy, once the store has read it)
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            *posp = final_pos;
            bulk_store(gst, cur, BYTES);
            bulk_commit();
            const long long gj = take();
            s_next = gj;
            if constexpr (IP) bulk_wait_read();
            if (gj < a.gens) {
                mbar_arrive_expect_tx(&bar, BYTES);
                bulk_load(nxt, state_of(gj), BYTES, &bar);
            }
            bulk_wait_read();   // `cur` may be overwritten once the store has read it
        }
        if constexpr (!IP) cb ^= 1;
        __syncthreads();
        gi = s_next;
    }
    if (tid == 0) bulk_wait_all();
}

template <class G, int M, int VW, int T, bool IP, class P, bool UNITS>
static cudaError_t launch_mt_pu(const GenArgs& a, cudaStream_t st)
{
    constexpr int smem = (IP ? 1 : 2) * G::N * M * static_cast<int>(sizeof(typename G::W));
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(gen_mt_kernel<G, M, VW, T, IP, P, UNITS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // unit launches are persistent: a few CTAs per SM pull units from the counter
    long long grid = a.gens < (1LL << 30) ? a.gens : (1LL << 30);
    if (UNITS && a.work_counter && !a.cta_per_unit) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long persistent = static_cast<long long>(sms) * mt_ctas_per_sm<G, M, T, IP>();
        if (grid > persistent) grid = persistent;
    }
    gen_mt_kernel<G, M, VW, T, IP, P, UNITS><<<static_cast<unsigned>(grid), T, smem, st>>>(a);
    return cudaGetLastError();
}

template <class G, int M, int VW, int T, bool IP, class P>
static cudaError_t launch_mt_p(const GenArgs& a, cudaStream_t st)
{
    if (a.units) return launch_mt_pu<G, M, VW, T, IP, P, true>(a, st);
    return launch_mt_pu<G, M, VW, T, IP, P, false>(a, st);
}

// policy dispatch: typed kernels for the common type patterns, generic otherwise
template <class G, int M, int VW, int T, bool IP = false>
static cudaError_t launch_mt(const GenArgs& a, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    if constexpr (M >= 4) {
        const int d0 = a.seg[0].dtype, d1 = a.nseg > 1 ? a.seg[1].dtype : -1;
        if constexpr (sizeof(typename G::W) == 4) {
            if (a.nseg == 1 && d0 == VMT_U32) return launch_mt_p<G, M, VW, T, IP, Pol<VMT_U32, -1>>(a, st);
            if (a.nseg == 1 && d0 == VMT_F32) return launch_mt_p<G, M, VW, T, IP, Pol<VMT_F32, -1>>(a, st);
            if (a.nseg == 1 && d0 == VMT_F64) return launch_mt_p<G, M, VW, T, IP, Pol<VMT_F64, -1>>(a, st);
            if (a.nseg == 2 && d0 == VMT_U32 && d1 == VMT_F32)
                return launch_mt_p<G, M, VW, T, IP, Pol<VMT_U32, VMT_F32>>(a, st);
        } else {
            if (a.nseg == 1 && d0 == VMT_U64) return launch_mt_p<G, M, VW, T, IP, Pol<VMT_U64, -1>>(a, st);
            if (a.nseg == 1 && d0 == VMT_F64) return launch_mt_p<G, M, VW, T, IP, Pol<VMT_F64, -1>>(a, st);
            if (a.nseg == 2 && d0 == VMT_U64 && d1 == VMT_F64)
                return launch_mt_p<G, M, VW, T, IP, Pol<VMT_U64, VMT_F64>>(a, st);
        }
    }
    return launch_mt_p<G, M, VW, T, IP, PolGeneric>(a, st);
}


// ---------------------------------------------------------------------------
// M = 1: one warp per generator
// ---------------------------------------------------------------------------
// A single-lane generator (the base generator's own stream) has only n - m
// independent words per phase, too few to share a CTA's threads between
// barriers.  Here a warp owns one generator: its two state copies (2 n words)
// in shared memory, phases of eq. stepnomod separated by __syncwarp, lane i
// handling words i, i + 32, ... and storing them coalesced (one output per
// generator word).
constexpr int kM1Warps = 8;

template <class G, int DT>
__device__ __forceinline__ void m1_store(char* out, long long e, typename G::W z)
{
    if constexpr (sizeof(typename G::W) == 4) {
        if constexpr (DT == VMT_U32) __stcs(reinterpret_cast<unsigned int*>(out) + e, z);
        else __stcs(reinterpret_cast<float*>(out) + e, f32_of_u32(z));
    } else {
        if constexpr (DT == VMT_U64) __stcs(reinterpret_cast<unsigned long long*>(out) + e, z);
        else if constexpr (DT == VMT_F64) __stcs(reinterpret_cast<double*>(out) + e, f64_of_u64(z));
        else __stcs(reinterpret_cast<float*>(out) + e, f32_of_u64(z));
    }
}

// new words [K0, K1) of the block: x_k from the old copy (cur) and, beyond
// the old copy, from the new one (nxt); call word e + k for k < hi
template <class G, int DT, int K0, int K1>
__device__ __forceinline__ void m1_phase(const typename G::W* __restrict__ cur, typename G::W* __restrict__ nxt,
                                         char* __restrict__ out, long long e, int hi, int lane, const ShiftK& sk)
{
    constexpr int N = G::N, MM = G::MM;
    // the two copies never alias, so the loads of several words can be
    // issued ahead of the stores (unrolled)
#pragma unroll 4
    for (int k = K0 + lane; k < K1; k += 32) {
        const typename G::W x = G::twist(cur[k], k + 1 < N ? cur[k + 1] : nxt[0], k + MM < N ? cur[k + MM] : nxt[k + MM - N]);
        nxt[k] = x;
        if (k < hi) m1_store<G, DT>(out, e + k, G::temper(x, sk));
    }
}

template <class G, int DT, bool UNITS>
__global__ void __launch_bounds__(kM1Warps * 32) gen_mt1_kernel(GenArgs a)
{
    using W = typename G::W;
    constexpr int N = G::N, NM = N - G::MM;
    static_assert(N <= 3 * NM, "at most three phases");
    __shared__ __align__(16) W bufs[kM1Warps][2][N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long cursor = static_cast<long long>(blockIdx.x) * kM1Warps + warp;
    auto take = [&]() -> long long {
        if (UNITS && a.work_counter) {
            int u = 0;
            if (lane == 0) u = atomicAdd(a.work_counter, 1);
            return static_cast<long long>(__shfl_sync(0xFFFFFFFFu, u, 0));
        }
        const long long u = cursor;
        cursor += static_cast<long long>(gridDim.x) * kM1Warps;
        return u;
    };
    constexpr int esize = (DT == VMT_U32 || DT == VMT_F32) ? 4 : 8;
    for (long long gi = take(); gi < a.gens; gi = take()) {
        W* gst;
        int* posp;
        long long total;
        char* out;
        int p;
        if constexpr (UNITS) {
            const UnitDesc& ud = a.units[gi];
            gst = reinterpret_cast<W*>(ud.state);
            posp = ud.pos;
            total = ud.total;
            out = ud.out;
            p = *posp;
        } else {
            gst = reinterpret_cast<W*>(a.states) + gi * N;
            posp = a.pos_dev + gi;
            total = a.total;
            out = a.seg[0].out + (a.gen0 + gi) * a.seg[0].count * esize;
            p = a.pos;
        }
        W* cur = bufs[warp][0];
        W* nxt = bufs[warp][1];
        for (int k = lane; k < N; k += 32) cur[k] = gst[k];
        __syncwarp();
        long long e = 0;
        int final_pos = p;
        if (p < N && total > 0) {
            // rest of the current block: block word k is call word k - p
            const int hi = static_cast<int>(min(static_cast<long long>(N), p + total));
            for (int k = p + lane; k < hi; k += 32) m1_store<G, DT>(out, k - p, G::temper(cur[k], a.k));
            e = hi - p;
            final_pos = hi;
        }
        while (e < total) {
            const int hi = static_cast<int>(min(static_cast<long long>(N), total - e));
            m1_phase<G, DT, 0, NM>(cur, nxt, out, e, hi, lane, a.k);
            __syncwarp();
            m1_phase<G, DT, NM, (2 * NM < N ? 2 * NM : N)>(cur, nxt, out, e, hi, lane, a.k);
            __syncwarp();
            if constexpr (2 * NM < N) {
                m1_phase<G, DT, (2 * NM < N ? 2 * NM : N), N>(cur, nxt, out, e, hi, lane, a.k);
                __syncwarp();
            }
            W* t = cur;
            cur = nxt;
            nxt = t;
            e += hi;
            final_pos = hi;
        }
        for (int k = lane; k < N; k += 32) gst[k] = cur[k];
        if (lane == 0) *posp = final_pos;
        __syncwarp();
    }
}

template <class G, int DT, bool UNITS>
static cudaError_t launch_mt1_t(const GenArgs& a, cudaStream_t st)
{
    long long grid = (a.gens + kM1Warps - 1) / kM1Warps;
    if (UNITS && a.work_counter && !a.cta_per_unit) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long persistent = static_cast<long long>(sms) * 5;   // 40 KB of shared memory per CTA
        if (grid > persistent) grid = persistent;
    }
    if (grid > (1LL << 30)) grid = 1LL << 30;
    gen_mt1_kernel<G, DT, UNITS><<<static_cast<unsigned>(grid), kM1Warps * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <class G, int DT>
static cudaError_t launch_mt1(const GenArgs& a, cudaStream_t st)
{
    if (a.gens <= 0) return cudaSuccess;
    return a.units ? launch_mt1_t<G, DT, true>(a, st) : launch_mt1_t<G, DT, false>(a, st);
}


// the translation unit's flag: 1 if one of its kernels gave up on a bounded
// wait since the last reset (-1 if it could not be read)
static int read_timeout_flag(bool reset)
{
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_gen_timeout, sizeof(int)) != cudaSuccess) return -1;
    if (reset && v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_gen_timeout, &z, sizeof(int));
    }
    return v;
}

}  // namespace dev
}  // namespace vmt
