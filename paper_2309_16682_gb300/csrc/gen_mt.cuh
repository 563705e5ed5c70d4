// gen_mt.cuh -- store and output-plan helpers of the MT generation kernels
// (gen_mt.cu: the phase form; gen_mtc.cu: the chain form).
//
// A vector is VW consecutive native words of one row of X-hat (VW lanes).
// Tempered vectors are routed to their output segment by a plan made once per
// block: a typed plan when the call's output types are known at compile time
// (one segment, or two split at a run-time boundary), a generic plan (one
// segment per warp lane, resolved by shuffles) otherwise.
#pragma once
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

// Bytes of output per native word for an output type: 32-bit words give 4
// (u32, f32, and u64/f64 built from two words); 64-bit words give 8 (u64,
// f64) or 4 (f32).
template <typename W>
__device__ __forceinline__ int bytes_per_word(int dt)
{
    return (sizeof(W) == 4 || dt == VMT_F32) ? 4 : 8;
}

// Output plan of one block, spread over the lanes of every warp: lane s holds
// segment s (base address such that block word f goes to base + f * bpw, and
// its output type); every lane holds the block-coordinate segment boundaries.
// A 16-byte vector at block word f0 then needs three compares and two shuffles
// to find its segment and address.
struct BlockPlan {
    long long my_base;
    int my_dt;
    int b1, b2, b3;
    bool fast;   // every segment base aligned to a vector and every boundary on a vector

    template <class P, typename W, int VW>
    __device__ __forceinline__ void make(const GenArgs& a, const Emitter& em, long long delta)
    {
        const int lane = threadIdx.x & 31;
        int bnd = 0x7FFFFFFF;
        bool ok = true;
        my_base = 0;
        my_dt = VMT_U32;
        if (lane < a.nseg) {
            const SegArg& sg = a.seg[lane];
            const int bpw = bytes_per_word<W>(sg.dtype);
            const int esz = (sg.dtype == VMT_U32 || sg.dtype == VMT_F32) ? 4 : 8;
            my_dt = sg.dtype;
            (void)esz;
            my_base = reinterpret_cast<long long>(em.elem0(lane)) + (delta - sg.wbeg) * bpw;
            ok = (my_base % (VW * bpw)) == 0;
            long long b = sg.wbeg - delta;   // block word where the segment starts
            if (b < -1) b = -1;
            if (b > (1LL << 30)) b = 1LL << 30;
            bnd = static_cast<int>(b);
            if (b > 0 && b < (1LL << 30) && (b % VW) != 0) ok = false;
        }
        fast = __all_sync(0xFFFFFFFFu, ok);
        b1 = __shfl_sync(0xFFFFFFFFu, bnd, 1);
        b2 = __shfl_sync(0xFFFFFFFFu, bnd, 2);
        b3 = __shfl_sync(0xFFFFFFFFu, bnd, 3);
        if (a.nseg < 2) b1 = 0x7FFFFFFF;
        if (a.nseg < 3) b2 = 0x7FFFFFFF;
        if (a.nseg < 4) b3 = 0x7FFFFFFF;
    }
};

// store VW tempered words at block word f0 (fast path; the whole vector is in
// range, in one segment and aligned).  Executed by all lanes of the warp (the
// shuffles need them); `doit` masks the store.
template <typename W, int VW>
__device__ __forceinline__ void plan_store(const BlockPlan& P, int f0, const W (&z)[VW], bool doit)
{
    const int s = (f0 >= P.b1) + (f0 >= P.b2) + (f0 >= P.b3);
    const long long base = __shfl_sync(0xFFFFFFFFu, P.my_base, s);
    const int dt = __shfl_sync(0xFFFFFFFFu, P.my_dt, s);
    if (!doit) return;
    if (sizeof(W) == 4) {
        const uint32_t* u = reinterpret_cast<const uint32_t*>(z);
        char* ptr = reinterpret_cast<char*>(base + 4LL * f0);
        if (VW == 4) {
            if (dt == VMT_U32) __stcs(reinterpret_cast<uint4*>(ptr), make_uint4(u[0], u[1 % VW], u[2 % VW], u[3 % VW]));
            else if (dt == VMT_F32)
                __stcs(reinterpret_cast<float4*>(ptr), make_float4(f32_of_u32(u[0]), f32_of_u32(u[1 % VW]),
                                                                   f32_of_u32(u[2 % VW]), f32_of_u32(u[3 % VW])));
            else if (dt == VMT_U64) {
                ulonglong2 v;
                v.x = static_cast<unsigned long long>(u[0]) | (static_cast<unsigned long long>(u[1 % VW]) << 32);
                v.y = static_cast<unsigned long long>(u[2 % VW]) | (static_cast<unsigned long long>(u[3 % VW]) << 32);
                __stcs(reinterpret_cast<ulonglong2*>(ptr), v);
            } else {
                double2 v;
                v.x = f64_of_pair(u[0], u[1 % VW]);
                v.y = f64_of_pair(u[2 % VW], u[3 % VW]);
                __stcs(reinterpret_cast<double2*>(ptr), v);
            }
        } else if (VW == 2) {
            if (dt == VMT_U32) __stcs(reinterpret_cast<uint2*>(ptr), make_uint2(u[0], u[1 % VW]));
            else if (dt == VMT_F32) __stcs(reinterpret_cast<float2*>(ptr), make_float2(f32_of_u32(u[0]), f32_of_u32(u[1 % VW])));
            else if (dt == VMT_U64)
                __stcs(reinterpret_cast<unsigned long long*>(ptr),
                       static_cast<unsigned long long>(u[0]) | (static_cast<unsigned long long>(u[1 % VW]) << 32));
            else __stcs(reinterpret_cast<double*>(ptr), f64_of_pair(u[0], u[1 % VW]));
        } else {
            if (dt == VMT_U32) __stcs(reinterpret_cast<uint32_t*>(ptr), u[0]);
            else if (dt == VMT_F32) __stcs(reinterpret_cast<float*>(ptr), f32_of_u32(u[0]));
        }
    } else {
        const unsigned long long* u = reinterpret_cast<const unsigned long long*>(z);
        if (dt == VMT_F32) {
            char* ptr = reinterpret_cast<char*>(base + 4LL * f0);
            if (VW == 2) __stcs(reinterpret_cast<float2*>(ptr), make_float2(f32_of_u64(u[0]), f32_of_u64(u[1 % VW])));
            else __stcs(reinterpret_cast<float*>(ptr), f32_of_u64(u[0]));
        } else {
            char* ptr = reinterpret_cast<char*>(base + 8LL * f0);
            if (VW == 2) {
                if (dt == VMT_U64) {
                    ulonglong2 v;
                    v.x = u[0];
                    v.y = u[1 % VW];
                    __stcs(reinterpret_cast<ulonglong2*>(ptr), v);
                } else {
                    double2 v;
                    v.x = f64_of_u64(u[0]);
                    v.y = f64_of_u64(u[1 % VW]);
                    __stcs(reinterpret_cast<double2*>(ptr), v);
                }
            } else {
                if (dt == VMT_U64) __stcs(reinterpret_cast<unsigned long long*>(ptr), u[0]);
                else __stcs(reinterpret_cast<double*>(ptr), f64_of_u64(u[0]));
            }
        }
    }
}

// Emit the vector of VW tempered words at block word f0 whose valid block
// range is [lo, hi); delta converts block words to call words.
template <typename W, int VW>
__device__ __forceinline__ void emit_vec(const BlockPlan& P, const Emitter& em, int f0, const W (&z)[VW], int lo,
                                         int hi, long long delta, bool active)
{
    const bool full = active && f0 >= lo && f0 + VW <= hi;
    if (P.fast) {
        plan_store<W, VW>(P, f0, z, full);
        if (full || !active) return;
    }
    if (active) emit_words<VW>(em, f0, z, lo, hi, delta + lo);
}

// Output policy: the output types of a call known at compile time (one
// segment, or two segments split at a run-time boundary), or GENERIC (any
// segment list, resolved per vector through BlockPlan).
template <int DT0_, int DT1_>
struct Pol {
    static constexpr int DT0 = DT0_, DT1 = DT1_;
    static constexpr bool generic = DT0_ < 0;
    static constexpr int nseg = generic ? 0 : (DT1_ < 0 ? 1 : 2);
};
using PolGeneric = Pol<-1, -1>;

// store VW words of one statically typed segment at base + f0 * bytes_per_word
template <int DT, typename W, int VW>
__device__ __forceinline__ void store_typed(long long base, int f0, const W (&z)[VW])
{
    if constexpr (sizeof(W) == 4) {
        const uint32_t* u = reinterpret_cast<const uint32_t*>(z);
        char* ptr = reinterpret_cast<char*>(base + 4LL * f0);
        if constexpr (VW == 4) {
            if constexpr (DT == VMT_U32) __stcs(reinterpret_cast<uint4*>(ptr), make_uint4(u[0], u[1], u[2], u[3]));
            if constexpr (DT == VMT_F32)
                __stcs(reinterpret_cast<float4*>(ptr),
                       make_float4(f32_of_u32(u[0]), f32_of_u32(u[1]), f32_of_u32(u[2]), f32_of_u32(u[3])));
            if constexpr (DT == VMT_U64) {
                ulonglong2 v;
                v.x = static_cast<unsigned long long>(u[0]) | (static_cast<unsigned long long>(u[1]) << 32);
                v.y = static_cast<unsigned long long>(u[2]) | (static_cast<unsigned long long>(u[3]) << 32);
                __stcs(reinterpret_cast<ulonglong2*>(ptr), v);
            }
            if constexpr (DT == VMT_F64) {
                double2 v;
                v.x = f64_of_pair(u[0], u[1]);
                v.y = f64_of_pair(u[2], u[3]);
                __stcs(reinterpret_cast<double2*>(ptr), v);
            }
        } else if constexpr (VW == 2) {
            if constexpr (DT == VMT_U32) __stcs(reinterpret_cast<uint2*>(ptr), make_uint2(u[0], u[1]));
            if constexpr (DT == VMT_F32)
                __stcs(reinterpret_cast<float2*>(ptr), make_float2(f32_of_u32(u[0]), f32_of_u32(u[1])));
            if constexpr (DT == VMT_U64)
                __stcs(reinterpret_cast<unsigned long long*>(ptr),
                       static_cast<unsigned long long>(u[0]) | (static_cast<unsigned long long>(u[1]) << 32));
            if constexpr (DT == VMT_F64) __stcs(reinterpret_cast<double*>(ptr), f64_of_pair(u[0], u[1]));
        }
    } else {
        const unsigned long long* u = reinterpret_cast<const unsigned long long*>(z);
        if constexpr (VW == 2) {
            if constexpr (DT == VMT_F32)
                __stcs(reinterpret_cast<float2*>(reinterpret_cast<char*>(base + 4LL * f0)),
                       make_float2(f32_of_u64(u[0]), f32_of_u64(u[1])));
            if constexpr (DT == VMT_U64) {
                ulonglong2 v;
                v.x = u[0];
                v.y = u[1];
                __stcs(reinterpret_cast<ulonglong2*>(reinterpret_cast<char*>(base + 8LL * f0)), v);
            }
            if constexpr (DT == VMT_F64) {
                double2 v;
                v.x = f64_of_u64(u[0]);
                v.y = f64_of_u64(u[1]);
                __stcs(reinterpret_cast<double2*>(reinterpret_cast<char*>(base + 8LL * f0)), v);
            }
        } else if constexpr (VW == 1) {
            if constexpr (DT == VMT_F32) __stcs(reinterpret_cast<float*>(reinterpret_cast<char*>(base + 4LL * f0)), f32_of_u64(u[0]));
            if constexpr (DT == VMT_U64) __stcs(reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(base + 8LL * f0)), u[0]);
            if constexpr (DT == VMT_F64) __stcs(reinterpret_cast<double*>(reinterpret_cast<char*>(base + 8LL * f0)), f64_of_u64(u[0]));
        }
    }
}

// Per-block plan for a static policy: segment bases and the boundary in block
// words; ok when both bases are vector-aligned and the boundary falls on a vector.
struct TypedPlan {
    long long base0, base1;
    int b1;
    bool ok;

    template <class P, typename W, int VW>
    __device__ __forceinline__ void make(const GenArgs& a, const Emitter& em, long long delta)
    {
        const int bpw0 = bytes_per_word<W>(P::DT0);
        base0 = reinterpret_cast<long long>(em.elem0(0)) + (delta - a.seg[0].wbeg) * bpw0;
        ok = (base0 % (VW * bpw0)) == 0;
        b1 = 0x7FFFFFFF;
        base1 = 0;
        if constexpr (P::nseg == 2) {
            const int bpw1 = bytes_per_word<W>(P::DT1);
            base1 = reinterpret_cast<long long>(em.elem0(1)) + (delta - a.seg[1].wbeg) * bpw1;
            ok = ok && (base1 % (VW * bpw1)) == 0;
            long long b = a.seg[1].wbeg - delta;
            if (b < -1) b = -1;
            if (b > (1LL << 30)) b = 1LL << 30;
            b1 = static_cast<int>(b);
            if (b > 0 && b < (1LL << 30) && (b % VW) != 0) ok = false;
        }
    }
};

template <class P>
struct PlanOf {
    using type = TypedPlan;
};
template <>
struct PlanOf<PolGeneric> {
    using type = BlockPlan;
};

// Emit the vector at block word f0 (valid block range [lo, hi); block word f
// is call word f + delta).  `check` is false when the whole vector is known to
// be in range.  All lanes call this (the generic plan shuffles).
template <class P, typename W, int VW>
__device__ __forceinline__ void emit_p(const typename PlanOf<P>::type& plan, const Emitter& em, int f0,
                                       const W (&z)[VW], int lo, int hi, long long delta, bool active, bool check)
{
    const bool full = active && (!check || (f0 >= lo && f0 + VW <= hi));
    if constexpr (P::generic) {
        if (plan.fast) {
            plan_store<W, VW>(plan, f0, z, full);
            if (full || !active) return;
        }
        if (active) emit_words<VW>(em, f0, z, lo, hi, delta + lo);
    } else {
        if (full && plan.ok) {
            if (P::nseg == 1 || f0 < plan.b1) store_typed<P::DT0, W, VW>(plan.base0, f0, z);
            else store_typed<(P::nseg == 2 ? P::DT1 : P::DT0), W, VW>(plan.base1, f0, z);
        } else if (active) {
            emit_words<VW>(em, f0, z, lo, hi, delta + lo);
        }
    }
}

}  // namespace dev
}  // namespace vmt
