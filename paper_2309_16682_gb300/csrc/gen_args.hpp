// gen_args.hpp -- launch arguments of the generation kernels (gen_mt.cu,
// gen_sfmt.cuh) and the block geometry of the three generators.  Kept apart
// from vmt_internal.hpp so that the generation kernels depend on this file
// only.
#pragma once
#include <cstdint>

#include "../../include/vmt.h"

#define VMT_MAXSEG 4

namespace vmt {

// Block sizes in native words (u32 for MT19937-32 and SFMT19937, u64 for
// MT19937-64): n * M * (u32 per unit).
inline int units_per_lane(int variant) { return variant == VMT_MT19937_32 ? 624 : (variant == VMT_MT19937_64 ? 312 : 156); }
inline int words_per_unit(int variant) { return variant == VMT_SFMT19937 ? 4 : 1; }
inline int word_bytes(int variant) { return variant == VMT_MT19937_64 ? 8 : 4; }
inline int64_t block_words(int variant, int lanes) { return static_cast<int64_t>(units_per_lane(variant)) * lanes * words_per_unit(variant); }
inline int64_t state_bytes_per_gen(int variant, int lanes) { return block_words(variant, lanes) * word_bytes(variant); }

// One output segment of a generate call.  Generator g writes its outputs of
// this segment at out + g*count elements; the segment covers call-relative
// native words [wbeg, wend).
struct SegArg {
    char* out;
    long long count;
    long long wbeg, wend;
    int dtype;
    int fast;  // out and count*elem_size are multiples of 16 bytes
};

// One unit of a ragged or batched launch: one generator with its own state,
// stream position, length and output (a single segment of type seg[0].dtype).
struct UnitDesc {
    char* state;         // X-hat of the generator
    int* pos;            // its block position (read at start, written at end)
    long long total;     // native words to produce
    char* out;           // first output element
};

// Compiled configurations of the MT generation kernels, per (variant, lanes);
// the first row of a (variant, lanes) group is its default.  form: kPhase = one CTA per
// generator, all threads on each phase of eq. (stepnomod), a barrier between
// phases (gen_mt.cu); kChain = a thread owns a chain of rows j, j+(n-m),
// j+2(n-m), one barrier per block, a CTA owns lpc of the M lanes (gen_mtc*.cu);
// kInPlace = the phase form on one copy of X-hat (gen_mt.cu).
// store = bytes per vector store (16 or 8).
enum { kPhase = 0, kChain = 1, kInPlace = 2 };
struct KernelCfg {
    int variant, lanes, form, lpc, threads, store;
};
constexpr KernelCfg kKernelCfgs[] = {
    // V-MT19937-32
    {VMT_MT19937_32, 16, kInPlace, 16, 256, 16},
    {VMT_MT19937_32, 16, kPhase, 16, 512, 16},
    {VMT_MT19937_32, 16, kPhase, 16, 1024, 16},
    {VMT_MT19937_32, 16, kChain, 8, 256, 16},
    {VMT_MT19937_32, 16, kChain, 16, 512, 16},
    {VMT_MT19937_32, 16, kChain, 8, 128, 16},
    {VMT_MT19937_32, 16, kChain, 8, 256, 8},
    {VMT_MT19937_32, 8, kInPlace, 8, 256, 16},
    {VMT_MT19937_32, 8, kPhase, 8, 256, 16},
    {VMT_MT19937_32, 8, kPhase, 8, 512, 16},
    {VMT_MT19937_32, 8, kChain, 8, 256, 16},
    {VMT_MT19937_32, 8, kChain, 8, 128, 16},
    {VMT_MT19937_32, 4, kPhase, 4, 256, 16},
    {VMT_MT19937_32, 4, kChain, 4, 128, 16},
    // V-MT19937-64
    {VMT_MT19937_64, 16, kInPlace, 16, 256, 16},
    {VMT_MT19937_64, 16, kPhase, 16, 512, 16},
    {VMT_MT19937_64, 16, kPhase, 16, 1024, 16},
    {VMT_MT19937_64, 16, kChain, 4, 160, 16},
    {VMT_MT19937_64, 16, kChain, 8, 320, 16},
    {VMT_MT19937_64, 8, kInPlace, 8, 256, 16},
    {VMT_MT19937_64, 8, kPhase, 8, 256, 16},
    {VMT_MT19937_64, 8, kPhase, 8, 512, 16},
    {VMT_MT19937_64, 8, kChain, 4, 160, 16},
    {VMT_MT19937_64, 8, kChain, 8, 320, 16},
    {VMT_MT19937_64, 8, kChain, 4, 160, 8},
    {VMT_MT19937_64, 4, kInPlace, 4, 256, 16},
    {VMT_MT19937_64, 4, kPhase, 4, 256, 16},
    {VMT_MT19937_64, 4, kChain, 4, 160, 16},
};
constexpr int kNumKernelCfgs = static_cast<int>(sizeof(kKernelCfgs) / sizeof(kKernelCfgs[0]));

// row of the table for candidate `index` of (variant, lanes), or nullptr
inline const KernelCfg* kernel_cfg(int variant, int lanes, int index)
{
    int k = 0;
    for (int i = 0; i < kNumKernelCfgs; ++i)
        if (kKernelCfgs[i].variant == variant && kKernelCfgs[i].lanes == lanes) {
            if (k == index) return &kKernelCfgs[i];
            ++k;
        }
    return nullptr;
}

inline int kernel_cfg_count(int variant, int lanes)
{
    int k = 0;
    for (int i = 0; i < kNumKernelCfgs; ++i) k += kKernelCfgs[i].variant == variant && kKernelCfgs[i].lanes == lanes;
    return k;
}

// Multipliers 2^s for the left shifts of the tempering (see vmt_device.cuh):
// kernel parameters, set by every launch of the MT generation kernels.
struct ShiftK {
    uint32_t p7, p15, p17, p5;
};
constexpr ShiftK kShiftK{1u << 7, 1u << 15, 1u << 17, 1u << 5};

struct GenArgs {
    void* states;      // [gens][block words] (lock-step mode)
    long long gens;    // generators (lock-step) or units (unit mode) in the launch
    long long gen0;    // first generator's index in the output arrays (lock-step mode)
    int pos;           // lock-step mode: the block position shared by all generators
    int* pos_dev;      // lock-step mode: per-generator block positions, written at end
    long long total;   // native words per generator in this call (lock-step mode)
    int nseg;
    SegArg seg[VMT_MAXSEG];
    int kcfg;          // kernel configuration: candidate index of (variant, lanes) in kKernelCfgs (0: default)
    const UnitDesc* units;   // unit mode when non-null: one entry per unit, longest first
    int* work_counter;       // unit mode: next unit = atomicAdd(work_counter, 1) (zeroed before launch)
    ShiftK k;                // tempering multipliers (set by the MT launchers)
    int cta_per_unit;        // unit mode: one CTA per unit instead of a persistent grid, so that CTAs of
                             // other (higher-priority) streams get an SM whenever a unit finishes
};

}  // namespace vmt
