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

struct GenArgs {
    void* states;      // [gens][block words] (lock-step mode)
    long long gens;    // generators (lock-step) or units (unit mode) in the launch
    long long gen0;    // first generator's index in the output arrays (lock-step mode)
    int pos;           // lock-step mode: the block position shared by all generators
    int* pos_dev;      // lock-step mode: per-generator block positions, written at end
    long long total;   // native words per generator in this call (lock-step mode)
    int nseg;
    SegArg seg[VMT_MAXSEG];
    int threads;       // CTA size among the compiled ones (0: default), set by the tuning table
    const UnitDesc* units;   // unit mode when non-null: one entry per unit, longest first
    int* work_counter;       // unit mode: next unit = atomicAdd(work_counter, 1) (zeroed before launch)
};

}  // namespace vmt
