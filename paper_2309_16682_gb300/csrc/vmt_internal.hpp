// vmt_internal.hpp -- launch descriptors shared by the C-ABI layer and the
// CUDA kernels.  Not part of the public interface (include/vmt.h is).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

#include <vector>

#include "../../include/vmt.h"

#include "gen_args.hpp"

namespace vmt {

// Jump work item: dst = c(F) src for one lane-state.  Unit u of the source
// state lives at src + u*src_stride units (a unit is one word, or one 128-bit
// element for SFMT19937); likewise for dst.  src and dst may alias.
struct JumpItem {
    const void* src;
    void* dst;
    int src_stride;
    int dst_stride;
    int poly;      // row of the polynomial table
    int deg;       // degree of that polynomial (-1: zero polynomial)
};

constexpr int kPolyWords = 640;  // u32 words per polynomial row (20480 bits)

// Jump work items described by a formula instead of a list (so that
// initialisation needs no host-built arrays):
//   kFanOut: item g*lanes + t writes lane t of generator g's X-hat as
//            row t*16/lanes applied to g's base state (unit-major base);
//   kDigit:  item g applies row 16 + 255*digit + d - 1 in place to g's base
//            state, d = byte `digit` of jumps[g] (nothing when d = 0).
//   kChunk:  item k*lanes + t writes lane t of chunk state k (X-hat layout in
//            `states`) as row chunk_row0 + c - 1 applied to lane t of request r's
//            X-hat (in `base`, X-hat layout), (r, c) = chunk_map[k].
struct JumpGrid {
    enum { kFanOut = 1, kDigit = 2, kChunk = 3 };
    int mode;
    long long count;
    int lanes;
    char* base;
    int unit_bytes;
    char* states;
    long long gen_bytes;
    const unsigned long long* jumps;
    int digit;
    const int* row_deg;
    const int2* chunk_map;
    int chunk_row0;
    // run-time recurrence of a twisted GFSR (eq. step with user parameters):
    // x_{k+n} = x_{k+m} ^ (y >> 1) ^ (y odd ? a : 0), y = (x_k & upper) | (x_{k+1} & lower)
    unsigned tg_m, tg_upper, tg_lower, tg_a;
};

// Chunks of one long stream: chunk c starts at S word c * chunk_words(...)
// (a whole number of blocks), so its lanes are the stream's lanes advanced by
// c * kChunkBlocks * n steps.  Rows for c = 1 .. kChunkRows of that jump are
// kept per variant.
constexpr int kChunkBlocks = 1024;
constexpr int kChunkRows = 255;
inline int64_t chunk_words(int variant, int lanes) { return static_cast<int64_t>(kChunkBlocks) * block_words(variant, lanes); }

// jump of twisted GFSR states (n words each, compiled n only): items' src/dst
// point at the states, the grid carries the recurrence; cta = one CTA per
// lane-jump (else one warp); cudaErrorNotSupported for an n not compiled
constexpr int kTgfsrSizes[] = {4, 5, 17};
cudaError_t launch_tgfsr_jump(int n, bool cta, const JumpItem* items, long long nitems, const JumpGrid& gr,
                              const uint32_t* polys, cudaStream_t s);

// ragged: generators of one launch may differ in position or length
cudaError_t launch_generate(int variant, int lanes, const GenArgs& a, bool ragged, cudaStream_t s);
// the pass schedule of MT kernel configuration `index` (see vmt_tune_pass_cut);
// -1 for a chain-form or missing configuration
int pass_cut(int variant, int lanes, int index, int* out8);
cudaError_t launch_seed(int variant, long long count, const unsigned long long* seeds, void* base, cudaStream_t s);
// shared (for launches that share the GPU with long-running kernels, the
// server's initialisation), whatever the count: 1 every lane-jump on a
// four-warp CTA with a ~20 KB ring; 0 the default choice
constexpr int kJumpShared = 1;   // the form the server uses
cudaError_t launch_jump(int variant, const JumpItem* items, long long nitems, const uint32_t* polys, cudaStream_t s,
                        int shared = 0);
cudaError_t launch_jump_grid(int variant, const JumpGrid& gr, long long nitems, const uint32_t* polys, cudaStream_t s,
                             int shared = 0);
cudaError_t launch_fill_int(int* p, long long n, int value, cudaStream_t s);
// jump launches of fewer items than `items` run one CTA per item
void set_jump_split_below(int variant, long long items);
long long get_jump_split_below(int variant);
// every jump launch of the variant in the shared form (1 compact; 0 off)
void set_jump_compact(int variant, int form);
int get_jump_compact(int variant);

}  // namespace vmt

// A set of `count` V-generators (the public handle of include/vmt.h).
struct vmt_state {
    int variant = 0;
    int lanes = 0;
    int64_t count = 0;
    std::vector<int64_t> h_pos;  // per generator: native words of its current block already emitted
    bool uniform = true;         // all h_pos equal
    int* d_pos = nullptr;        // device copy, read and written by the generation kernels
    void* d_states = nullptr;    // [count][block words]
    int device = 0;
    bool async_alloc = false;    // device memory from a stream-ordered pool
    // unit-launch scratch (ragged calls): pinned host staging and device copy
    vmt::UnitDesc* h_units = nullptr;
    vmt::UnitDesc* d_units = nullptr;
    int* d_counter = nullptr;
    int64_t units_cap = 0;
    cudaEvent_t units_free = nullptr;   // recorded after the last upload of h_units
};

namespace vmt {

// one launch over a unit table already on the device; n units of the given
// kernel, scheduled through counter (zeroed here), longest first.  Persistent
// (a few CTAs per SM) by default; cta_per_unit gives each unit its own CTA.
int launch_unit_table(int variant, int lanes, int dtype, const UnitDesc* d_units, int64_t n, int* counter,
                      void* stream, bool cta_per_unit = false);

// stream-ordered allocation from `pool`, or from the device's default pool
// when pool is null
inline cudaError_t malloc_async(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t s)
{
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, s) : cudaMallocAsync(p, bytes, s);
}

// state creation with optional stream-ordered allocation (from `pool` when
// given), and its release
int init_batch_impl(vmt_state** out, int variant, int lanes, int64_t count, const uint64_t* seeds,
                    const uint64_t* jumps, void* cuda_stream, bool async_alloc, cudaMemPool_t pool = nullptr);
// several objects of one variant: seeding and offsets once, fan-out per object
int init_multi_impl(vmt_state** outs, int variant, int nsub, const int* lanes, const int64_t* counts,
                    const uint64_t* seeds, const uint64_t* jumps, void* cuda_stream, bool async_alloc,
                    cudaMemPool_t pool = nullptr, int shared_jumps = 0);
void free_state_async(vmt_state* st, void* cuda_stream);

// `count` generators with unset states (to be written by a jump), fresh
// positions, stream-ordered memory
int alloc_states_async(vmt_state** out, int variant, int lanes, int64_t count, void* cuda_stream,
                       cudaMemPool_t pool = nullptr);

// chunk states: chunk k = row (chunk_map[k].y) applied to every lane of
// request chunk_map[k].x of `requests`; d_map on the device
int launch_chunk_jumps(const vmt_state* requests, vmt_state* chunks, const int2* d_map, void* cuda_stream,
                       int shared_jumps = 0);

// tuned kernel configuration of a (variant, lanes) pair: an index into that
// pair's rows of kKernelCfgs (0: the default)
int tuned_kcfg(int variant, int lanes);

// 1 if a generation kernel gave up on a bounded wait (and reset the flag when asked)
int read_generate_timeout(bool reset);

// message returned by vmt_last_error() on this thread
void set_last_error(const char* msg);

}  // namespace vmt
