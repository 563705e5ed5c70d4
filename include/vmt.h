/*
 * vmt.h -- C ABI of the GB300 V-family generator library (libvmt.so).
 *
 * The V-family of arXiv 2309.16682 ("VMT19937: A SIMD-Friendly Pseudo Random
 * Number Generator based on Mersenne Twister 19937"), Sec. 3: M instances of a
 * base generator (MT19937-32, MT19937-64 or SFMT19937) are de-phased by
 * jump-ahead so that lane t starts J = ceil(P/M) = 2^(19937 - log2 M) steps
 * after lane t-1 (Table "jvalues"), and their outputs are polled round robin
 * into one stream S (eq. combseq): S[kM + t] = z_{tJ + k}.  For SFMT19937 the
 * interleave unit is the 128-bit element, emitted as four 32-bit words,
 * least-significant sub-word first.
 *
 * Conventions for every call:
 *   - return 0 (VMT_OK) or a negative VMT_E* code; vmt_last_error() gives a
 *     thread-local message for the last failure on the calling thread;
 *   - `cuda_stream` is a cudaStream_t (NULL = legacy default stream); device
 *     work is enqueued on it and the call returns without synchronising unless
 *     the call's description says otherwise;
 *   - a vmt_state owns its device memory until vmt_free(); device pointers
 *     passed in (out_dev) are owned by the caller;
 *   - all generators of one vmt_state advance in lock-step: every generate call
 *     takes the same number of words from each of them.
 *
 * Words: "native words" are 32-bit for MT19937-32 and SFMT19937 and 64-bit for
 * MT19937-64.  Output types and the words they consume:
 *   VMT_U32  one 32-bit word                 (not defined for MT19937-64)
 *   VMT_U64  a | b << 32 from two 32-bit words a, b (32-bit variants), or one
 *            64-bit word
 *   VMT_F32  (z >> 8) * 2^-24 from a 32-bit word, (z >> 40) * 2^-24 from a
 *            64-bit word; in [0, 1), exact
 *   VMT_F64  ((a >> 5) * 2^26 + (b >> 6)) * 2^-53 from two 32-bit words, or
 *            (z >> 11) * 2^-53 from a 64-bit word; in [0, 1), exact
 * The conversions are not in the paper; they are the usual 24/53-bit forms.
 */
#ifndef VMT_H
#define VMT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* base generators (Sec. 2.2, 2.3, 2.4) */
#define VMT_MT19937_32 0
#define VMT_MT19937_64 1
#define VMT_SFMT19937 2

/* output types */
#define VMT_U32 0
#define VMT_U64 1
#define VMT_F32 2
#define VMT_F64 3

/* status codes */
#define VMT_OK 0
#define VMT_EINVAL (-1)   /* bad argument (variant, lanes, dtype, size, pointer) */
#define VMT_ENOMEM (-2)   /* device or host allocation failed */
#define VMT_ECUDA (-3)    /* a CUDA runtime call failed */
#define VMT_ETIMEOUT (-4) /* a bounded wait ran out */
#define VMT_EBUSY (-5)    /* resource in use / admission refused */
#define VMT_ESTATE (-6)   /* corrupt or mismatching exported state */

typedef struct vmt_state vmt_state;

/*
 * vmt_init -- create one V-family generator (Sec. 3, construction of the
 * V generator; Sec. 3.1, initialisation by jump-ahead).
 *   st        out: the new generator (free with vmt_free)
 *   variant   VMT_MT19937_32, VMT_MT19937_64 or VMT_SFMT19937
 *   lanes     M in {1, 2, 4, 8, 16}
 *   seed      base-generator seed (32-bit variants use seed mod 2^32); seeding
 *             follows the C++ standard's mersenne_twister_engine recurrence,
 *             SFMT19937 adds its period certification
 *   jump      offset d applied to the base state before de-phasing: lane t
 *             starts at z_{d + tJ}
 * The first call for a variant in a process computes (or loads from the
 * on-disk cache) the variant's minimal polynomial and jump polynomials; this
 * takes seconds once and synchronises `cuda_stream`.
 */
int vmt_init(vmt_state** st, int variant, int lanes, uint64_t seed, uint64_t jump, void* cuda_stream);

/*
 * vmt_init_batch -- `count` independent V-family generators in one state
 * object (same variant and M).  seeds[g] and jumps[g] (host arrays, copied;
 * jumps may be NULL for all-zero) set generator g as in vmt_init.  Seeding,
 * jump-ahead and lane de-phasing run as batched kernels.
 */
int vmt_init_batch(vmt_state** st, int variant, int lanes, int64_t count, const uint64_t* seeds,
                   const uint64_t* jumps, void* cuda_stream);

/*
 * vmt_jump -- apply the jump polynomial c(F) to every lane of every generator
 * (Sec. 3.1).  poly: host array of ceil(nbits/64) words, bit i of word i/64 is
 * the coefficient of x^i; nbits <= 20480.  A polynomial congruent to x^d
 * modulo the minimal polynomial advances every lane by d steps.
 */
int vmt_jump(vmt_state* st, const uint64_t* poly, int64_t nbits, void* cuda_stream);

/*
 * vmt_jump_poly -- write x^(d * 2^log2_extra) mod mu into poly_out (host,
 * cap_words uint64 words).  mu is the variant's minimal polynomial.  Returns
 * the number of words written, or a negative status.  With d = 1 and
 * log2_extra = 19937 - log2 M it gives the lane spacing J of Table "jvalues".
 */
int vmt_jump_poly(int variant, uint64_t d, int log2_extra, uint64_t* poly_out, int64_t cap_words);

/*
 * vmt_prepare -- build, for the current device, every table the variant's
 * initialisation and jumps use: the characteristic polynomial (Sec. 3.1.2,
 * found by Berlekamp-Massey or read from the cache directory), the chain
 * x^(2^q) mod it, the base-256 digit rows x^(v 256^i) of 64-bit jump offsets
 * and the rows x^(c * 1024 * n) that cut long server requests into chunks.
 * Every other entry point builds what it needs on first use; calling this
 * first moves that one-time cost (up to seconds) out of the first request.
 * Returns VMT_EINVAL for a bad variant.
 */
int vmt_prepare(int variant, void* cuda_stream);

/*
 * vmt_generate -- the next n outputs of type dtype from every generator.
 * Generator g writes out_dev[g*n .. g*n + n) (device memory, caller-owned,
 * at least count*n elements).  The stream continues across calls: a call
 * resumes exactly at the next word of S.  n >= 0.
 */
int vmt_generate(vmt_state* st, int64_t n, int dtype, void* out_dev, void* cuda_stream);

/*
 * vmt_generate_multi -- several consecutive output segments in one pass:
 * segment i takes counts[i] outputs of type dtypes[i] from the stream, and
 * generator g writes them at outs[i] + g*counts[i] elements.  Equivalent to
 * nseg consecutive vmt_generate calls; 1 <= nseg <= 4.
 */
int vmt_generate_multi(vmt_state* st, int nseg, const int64_t* counts, const int* dtypes, void* const* outs,
                       void* cuda_stream);

/*
 * vmt_generate_ragged -- generator g takes the next n[g] outputs of type dtype
 * into the device buffer outs[g] (host arrays of count entries; n[g] may be 0).
 * Generators then sit at different stream positions; later calls continue
 * each one exactly.  All generators run in one persistent launch that hands
 * them to CTAs longest first.  Limits: n[g] * words-per-output <= 2^30, and
 * two-word outputs (u64/f64 from 32-bit generators) need an even stream
 * position and at least 2 lanes (VMT_EINVAL otherwise).
 */
int vmt_generate_ragged(vmt_state* st, const int64_t* n, int dtype, void* const* outs, void* cuda_stream);

/*
 * Batches: many state objects (any variants and lane counts) generating in
 * one pass.  vmt_batch_add(b, st, n, dtype, out) asks every generator g of st
 * for its next n outputs at out + g*n; a state may appear once per batch.
 * vmt_batch_run enqueues one persistent launch per (variant, lanes, dtype)
 * group, units longest first; vmt_batch_run_graph does the same through a
 * CUDA graph captured on its first call and replayed afterwards (the unit
 * table, output pointers and lengths are fixed at capture; the stream
 * positions advance on the device, so each replay continues every stream).
 * Adding items or vmt_batch_clear drops the graph.  Same limits as
 * vmt_generate_ragged.
 */
typedef struct vmt_batch vmt_batch;
int vmt_batch_create(vmt_batch** b);
int vmt_batch_add(vmt_batch* b, vmt_state* st, int64_t n, int dtype, void* out_dev);
int vmt_batch_run(vmt_batch* b, void* cuda_stream);
int vmt_batch_run_graph(vmt_batch* b, void* cuda_stream);
int vmt_batch_clear(vmt_batch* b);
void vmt_batch_destroy(vmt_batch* b);

/*
 * Serving (the paper has no counterpart; it serves the paper's generators to
 * many independent clients).  A request asks for n outputs of type dtype from
 * one fresh V-generator (variant, lanes, seed, jump as in vmt_init).  Requests
 * are admitted FIFO while two budgets hold: generator states of batches in
 * flight (state_budget_bytes) and outputs not yet released
 * (output_budget_bytes).  A worker thread launches admitted requests as soon
 * as they arrive, at most max_batch (1..4096) per batch: batched seeding and
 * jump-ahead on one stream, a persistent ragged generation (longest first) on
 * another, so a new batch's initialisation overlaps the previous batch's
 * generation.  Requests of at most 16,384 outputs whose bytes fit the express
 * budget (output_budget_bytes / 16) run only in express batches: one slot per
 * variant with the highest-priority streams, ahead of the queue; their
 * outputs count against the express budget instead of the output budget, and
 * they pass a waiting request only where it would still fit the state budget
 * afterwards.
 * Latency: the server runs up to 29 streams at once.  CUDA maps streams onto
 * CUDA_DEVICE_MAX_CONNECTIONS hardware work queues (8 unless set before the
 * process creates its CUDA context), and work of streams that share a queue
 * is serialised: with 8, small requests wait behind long requests' jump
 * chains.  Set it to 32 (the Python package does so on import when unset).
 *   vmt_server_submit   never blocks; *id names the request
 *   vmt_server_poll     status VMT_SERVER_QUEUED / RUNNING / DONE or a negative
 *                       VMT_E* code (that request failed; the server goes on);
 *                       when DONE, *out_dev is the device buffer (n elements)
 *                       and *latency_s the time from submit to completion
 *   vmt_server_wait     blocks until the request is done or failed, or returns
 *                       VMT_ETIMEOUT after timeout_ms
 *   vmt_server_release  frees the output (after the client's own work on it
 *                       has finished) and returns its bytes to the budget
 * Limits: n * words-per-output <= 2^30; u64/f64 from 32-bit generators need
 * lanes >= 2.  A request larger than a budget fails with VMT_ENOMEM.
 * Memory: states and outputs come from a stream-ordered pool owned by the
 * server that keeps up to both budgets' bytes between requests; with
 * reserve != 0 the pool takes that memory at creation (creation fails with
 * VMT_ENOMEM if the device cannot hold it), so admitted requests never wait
 * for the CUDA driver to map memory, and every variant's tables are prepared
 * (vmt_prepare) before the server accepts requests.
 * Counters: host_launch_s is the worker's host time spent issuing batches;
 * init_gpu_s sums, over finished batches, the device time from the start of
 * a batch's initialisation to its end (seeding, jumps, chunk jumps);
 * batch_gpu_s the device time from that start to the end of its generation.
 */
#define VMT_SERVER_QUEUED 0
#define VMT_SERVER_RUNNING 1
#define VMT_SERVER_DONE 2

typedef struct vmt_server vmt_server;
typedef struct {
    int64_t state_budget_bytes;
    int64_t output_budget_bytes;
    int max_batch;
    int reserve;   /* nonzero: map both budgets into the server's pool at creation */
} vmt_server_config;
typedef struct {
    int variant, lanes, dtype;
    uint64_t seed, jump;
    int64_t n;
} vmt_request;
typedef struct {
    int64_t queued, in_flight_batches, batches, completed, failed, bytes_out;
    int64_t state_bytes_in_use, output_bytes_in_use, peak_state_bytes, peak_output_bytes;
    double host_launch_s, init_gpu_s, batch_gpu_s;
    int64_t cancelled;
    /* express batches and their completed requests; sums over completed
     * requests of the time queued (submission to admission into a batch) and
     * of the time running (admission to completion), regular and express */
    int64_t express_batches, express_completed;
    double queued_s, running_s, express_queued_s, express_running_s;
    /* the express batches' share of init_gpu_s and batch_gpu_s */
    double express_init_gpu_s, express_batch_gpu_s;
} vmt_server_counters;

int vmt_server_create(vmt_server** s, const vmt_server_config* cfg);
int vmt_server_submit(vmt_server* s, const vmt_request* r, uint64_t* id);
int vmt_server_poll(vmt_server* s, uint64_t id, int* status, void** out_dev, int64_t* bytes, double* latency_s);
int vmt_server_wait(vmt_server* s, uint64_t id, int timeout_ms);
int vmt_server_release(vmt_server* s, uint64_t id);
/*
 * vmt_server_cancel -- withdraw a request that is still queued: its status
 * becomes VMT_ECANCELED (release it as any finished request).  VMT_EBUSY when
 * it is already running or finished, VMT_EINVAL for an unknown id.
 */
#define VMT_ECANCELED (-7)
/*
 * vmt_server_next_done -- completion queue: the id of the next request that
 * reached a final status (done, failed or cancelled), in the order they did,
 * each once; waits up to timeout_us microseconds and returns VMT_ETIMEOUT if
 * none came.  Requests released before they were taken from the queue are
 * skipped.
 */
int vmt_server_next_done(vmt_server* s, int64_t timeout_us, uint64_t* id);
int vmt_server_cancel(vmt_server* s, uint64_t id);
/*
 * Batched forms for clients with many requests in flight (one call and one
 * lock per batch instead of per request):
 *   vmt_server_submit_many   submits reqs[0..n) in order, ids[i] receiving
 *                            request i's id; all are checked first and
 *                            VMT_EINVAL submits none of them
 *   vmt_server_next_done_many  up to cap requests that reached a final status,
 *                            in completion order (as vmt_server_next_done),
 *                            with status[i] and latency_s[i] (submission to
 *                            completion, -1 unless done); waits up to
 *                            timeout_us for the first; returns the count
 *                            (0 when none came), or a negative error code
 *   vmt_server_release_many  vmt_server_release of each id; returns the first
 *                            error (the others are still released)
 */
int vmt_server_submit_many(vmt_server* s, const vmt_request* reqs, int64_t n, uint64_t* ids);
int64_t vmt_server_next_done_many(vmt_server* s, int64_t timeout_us, uint64_t* ids, int* status, double* latency_s,
                                  int64_t cap);
int vmt_server_release_many(vmt_server* s, const uint64_t* ids, int64_t n);
/*
 * vmt_server_inject -- host-side fault injection for tests: the next `count`
 * output allocations of the server fail as if device memory were exhausted
 * (VMT_INJECT_ALLOC).  Each such request fails alone with VMT_ENOMEM; the
 * rest of its batch and the server go on.  No GPU fault is involved.
 */
#define VMT_INJECT_ALLOC 1
int vmt_server_inject(vmt_server* s, int what, int count);
/* copy a finished request's output into host memory (cap bytes; synchronous) */
int vmt_server_copy(vmt_server* s, uint64_t id, void* host_buf, int64_t cap);
int vmt_server_stats(vmt_server* s, vmt_server_counters* stats);
void vmt_server_destroy(vmt_server* s);

/*
 * vmt_generate_host -- as vmt_generate but into host memory.  Pinned
 * (page-locked, device-mapped) memory is written directly by the generation
 * kernels; pageable memory through a device staging buffer in chunks, the
 * generation of one chunk overlapping the copy of the previous one.
 * Synchronises `cuda_stream` before returning.
 */
int vmt_generate_host(vmt_state* st, int64_t n, int dtype, void* out_host, void* cuda_stream);

/* Bytes of an exported state (header + all generators' states). */
int64_t vmt_state_bytes(const vmt_state* st);

/*
 * vmt_state_export / vmt_state_import -- checkpoint of every generator's
 * combined state X-hat (Sec. 3) and stream position.  export writes
 * vmt_state_bytes(st) bytes to host_buf (cap bytes available) and
 * synchronises; import overwrites a state object of the same variant, lanes
 * and count (VMT_ESTATE on mismatch).  A generator resumed from an export
 * continues the stream exactly.
 */
int vmt_state_export(const vmt_state* st, void* host_buf, size_t cap, void* cuda_stream);
int vmt_state_import(vmt_state* st, const void* host_buf, size_t len, void* cuda_stream);

/* Variant, lanes M, generator count and generator 0's current block position. */
int vmt_state_info(const vmt_state* st, int* variant, int* lanes, int64_t* count, int64_t* block_pos);

/* Device pointer of the combined states ([count][n][M] units) -- for tests. */
void* vmt_state_device_ptr(const vmt_state* st);

/*
 * vmt_device_status -- VMT_ETIMEOUT if, since the last reset, a generation
 * kernel gave up a bounded wait for one of its bulk copies (it then stops
 * without writing its outputs), VMT_OK otherwise.  Synchronises the device's
 * legacy stream.  reset != 0 clears the flag.
 */
int vmt_device_status(int reset);

/*
 * Tuning of the generation kernels (the paper has no counterpart: how a block
 * of eq. (stepnomod) is spread over a CTA is a GPU-specific choice).  Each
 * (variant, lanes) pair of MT19937-32/64 has a small list of compiled kernel
 * configurations, described by vmt_tune_kernels as four ints each:
 *   form           0: phase form -- one CTA per generator, two copies of
 *                     X-hat in shared memory, each pass of at most n-m rows
 *                     spread over all threads, a barrier between passes;
 *                     1: chain form -- a thread owns the rows j, j+(n-m),
 *                     j+2(n-m) of one column (one barrier per block);
 *                     2: in-place phase form -- one copy of X-hat, so more
 *                     CTAs share an SM (default for MT19937-32 with 8 or
 *                     16 lanes and MT19937-64 with 4, 8 or 16 lanes)
 *   lanes_per_cta  lanes of the generator one CTA owns (chain form: M/lanes
 *                     CTAs share a generator; unit launches use one CTA)
 *   threads        CTA size
 *   store_bytes    bytes per vector store (16 or 8)
 * Entry 0 is the default.  Every configuration gives identical output.  The
 * table starts at the defaults, can be preset with the environment variable
 * VMT_TUNE="mt32:16:1024,mt64:8:#2" (a phase-form CTA size, or #index), set
 * directly, or filled by the autotuner.
 *   vmt_tune_set       select the phase-form configuration with `threads`
 *                      threads (0: the default entry); VMT_EINVAL if none
 *   vmt_tune_get       CTA size of the selected configuration
 *   vmt_tune_kernels   writes min(count, cap) descriptions into desc
 *                      (4 * cap ints) and returns count
 *   vmt_tune_set_kernel / vmt_tune_get_kernel   select / read the index
 *   vmt_tune_pass_cut  the pass schedule of phase-form (0) or in-place (2)
 *                      configuration `index`, in units of vectors (VW lane
 *                      words of one row): out8 = {vectors per block, vectors
 *                      per pass, vectors per row, vectors in n-m rows,
 *                      vectors in m rows, threads, in place, early (the next
 *                      block's first-pass operands are loaded during the last
 *                      pass)}; VMT_EINVAL for the
 *                      chain form, SFMT19937 or an index out of range.  Needs
 *                      no GPU; tests check the schedule's hazards with it.
 *   vmt_autotune_grid  times every configuration on `count` generators
 *                      producing the caller's segment list (as
 *                      vmt_generate_multi: counts[i] outputs of dtypes[i] per
 *                      generator), two alternating rounds of `reps` timed
 *                      calls after a warm-up, each keeping its better mean;
 *                      writes min(count, cap) times (ms per call) into ms_out,
 *                      selects and returns the fastest in *best_index
 *   vmt_autotune[_multi]   the same, returning the winner's CTA size and time
 * SFMT19937 has one configuration.
 */
int vmt_tune_set(int variant, int lanes, int threads);
int vmt_tune_get(int variant, int lanes);
int vmt_tune_kernels(int variant, int lanes, int* desc, int cap);
int vmt_tune_pass_cut(int variant, int lanes, int index, int* out8);
int vmt_tune_set_kernel(int variant, int lanes, int index);
int vmt_tune_get_kernel(int variant, int lanes);
int vmt_autotune_grid(int variant, int lanes, int64_t count, int nseg, const int64_t* counts, const int* dtypes,
                      int reps, void* cuda_stream, double* ms_out, int cap, int* best_index);
/*
 * vmt_tune_save / vmt_tune_load -- the tuning table as a text file, one
 * "variant lanes form lanes_per_cta threads store_bytes" line per entry that
 * differs from the default (the autotuner's results can thus be kept per GPU
 * model and reapplied).  load also accepts "variant lanes threads" lines (a
 * phase-form CTA size), applies every valid line and returns VMT_EINVAL if a
 * line names a configuration that is not compiled (the valid ones still
 * apply) or the file cannot be read.
 */
int vmt_tune_save(const char* path);
int vmt_tune_load(const char* path);

/*
 * vmt_tune_jump_set / vmt_tune_jump_get -- jump launches (initialisation,
 * vmt_jump, server chunks) with fewer lane-jumps than split_below give each
 * lane-jump a whole CTA, whose warps share the work of one evaluation of
 * c(F) X (Sec. 3.1): lower latency, lower throughput.  Larger launches give
 * each lane-jump one warp.  0 never splits.  Results are identical either way.
 * The threshold is per variant; variant -1 sets all three.  get returns the
 * variant's threshold (VMT_EINVAL for a bad variant).
 */
int vmt_tune_jump_set(int variant, int64_t split_below);
int64_t vmt_tune_jump_get(int variant);
/*
 * vmt_tune_jump_compact -- on = 1: every jump launch of the variant (-1: all
 * three) uses the compact CTA form: four warps per lane-jump over a ~20 KB
 * ring of the sequence, extended in several rounds.  Each lane-jump is slower
 * than in the sixteen-warp CTA form, but a CTA needs little shared memory, so
 * it is scheduled next to long-running kernels of other streams (the server
 * always uses this form for its initialisation).  on = 0 returns to the
 * default choice, on = -1 only reads.  Returns the setting before the call
 * (1 or 0), or VMT_EINVAL.  Results are identical in every form.
 */
int vmt_tune_jump_compact(int variant, int on);

/*
 * vmt_stream_generate -- exact single-stream mode: the first n outputs, from
 * offset `jump`, of ONE base generator (MT19937-32, MT19937-64 or SFMT19937
 * as in Sec. 2, seeded as vmt_init with M = 1), i.e. the scalar generator's
 * own stream (std::mt19937, std::mt19937_64, SFMT19937's 32-bit output
 * sequence), written to out_dev (n elements).  It is produced in parallel:
 * the stream is cut into up to 2048 chunks of equal length, chunk j starting
 * from the base state jumped by j chunk lengths with the polynomial jump-ahead
 * of Sec. 3.1, and the chunks are generated concurrently.  `jump` counts
 * steps of the recurrence (SFMT: 128-bit elements, 4 outputs each).
 * dtype: VMT_U32 or VMT_F32 for the 32-bit generators; VMT_U64, VMT_F64 or
 * VMT_F32 for MT19937-64 (one output per generator word).  n <= 2^39.
 * Asynchronous on cuda_stream; all scratch is stream-ordered and released
 * before the call returns (in stream order).  VMT_EINVAL for a bad variant,
 * type, n or a null output.
 */
int vmt_stream_generate(int variant, uint64_t seed, uint64_t jump, int64_t n, int dtype, void* out_dev,
                        void* cuda_stream);

/*
 * Buffered scalar queries (the paper's scalar query mode, served from a
 * buffer; Sec. 4.4.1, scalar performance and optimised buffering).  One
 * V-generator (variant, lanes, seed, jump as in vmt_init) whose outputs of
 * type dtype are read one at a time on the host: the GPU's kernels write them
 * in bulk, buffer_outputs (1024 .. 2^28) at a time, directly into one of two
 * pinned, device-mapped host buffers while the host reads the other.  The sequence is exactly the
 * V-stream S that vmt_generate would return for the same generator.
 *   vmt_scalar_next   the next output (4 or 8 bytes) into *value
 *   vmt_scalar_take   the next n outputs into host memory
 *   vmt_scalar_drain  consumes `count` outputs one query at a time and returns
 *                     an order-sensitive checksum of them (measures the
 *                     per-query cost without a caller's loop)
 * Not thread-safe: one object per consuming thread.  Calls wait for a refill
 * only once every buffer_outputs outputs.  Errors: VMT_EINVAL, VMT_ENOMEM,
 * VMT_ECUDA; the restrictions of vmt_generate on dtype apply.
 */
typedef struct vmt_scalar vmt_scalar;
int vmt_scalar_create(vmt_scalar** q, int variant, int lanes, uint64_t seed, uint64_t jump, int dtype,
                      int64_t buffer_outputs);
int vmt_scalar_next(vmt_scalar* q, void* value);
int vmt_scalar_take(vmt_scalar* q, int64_t n, void* out_host);
int vmt_scalar_drain(vmt_scalar* q, int64_t count, uint64_t* checksum);
void vmt_scalar_destroy(vmt_scalar* q);

/*
 * vmt_measure_store_bw -- diagnostic, no paper counterpart: the device's HBM
 * write bandwidth as seen by a store-only kernel (16-byte streaming stores
 * over `bytes` bytes of a buffer it allocates and frees on cuda_stream), best
 * of `reps` timed launches per launch shape, in GB/s (10^9 bytes/s).  It is
 * the ceiling for kernels that mostly write.  Synchronises cuda_stream.
 * VMT_EINVAL for bytes < 1 MiB, reps < 1 or a null output; VMT_ENOMEM when
 * the buffer cannot be allocated.
 */
int vmt_measure_store_bw(int64_t bytes, int reps, double* best_gbs, void* cuda_stream);

/*
 * vmt_selftest_wait -- diagnostic, no paper counterpart: runs the bounded
 * mbarrier wait of the generation kernels on a barrier that nothing arrives
 * at, with a limit of limit_ns (1 us .. 10 s), on the device's legacy stream.
 * Returns VMT_ETIMEOUT when the wait gave up (the expected outcome; the
 * kernel then returns normally and the context stays usable), VMT_OK if it
 * did not, with the device-measured wait time in *elapsed_ns (may be null).
 * The generation kernels use a limit of one second per wait.
 */
int vmt_selftest_wait(int64_t limit_ns, int64_t* elapsed_ns);
int vmt_autotune(int variant, int lanes, int64_t count, int64_t n_per_gen, int dtype, int reps, void* cuda_stream,
                 int* best_threads, double* best_ms);
/* as vmt_autotune, timing vmt_generate_multi on the caller's own segment list
 * (the table is keyed by variant and lanes, so tune with the mix you run) */
int vmt_autotune_multi(int variant, int lanes, int64_t count, int nseg, const int64_t* counts, const int* dtypes,
                       int reps, void* cuda_stream, int* best_threads, double* best_ms);

/* Release a state object (NULL is allowed). */
void vmt_free(vmt_state* st);

/* Message for the last failing call on this thread ("" if none). */
const char* vmt_last_error(void);

/* Directory of the on-disk cache of minimal/jump polynomials (NULL: default). */
int vmt_set_cache_dir(const char* path);

/*
 * Host polynomial helpers (no GPU needed): Berlekamp-Massey, products modulo a
 * polynomial and the chain x^(2^q) mod mu, as used to build jump polynomials
 * (Sec. 3.1).  All polynomials are uint64 word arrays, bit i = coefficient of
 * x^i.
 *   vmt_poly_minpoly   bits: n sequence bits packed little-endian; writes
 *                      mu (cap_words) and returns deg mu (linear complexity)
 *   vmt_poly_mulmod    out = a * b mod mu (all nw words)
 *   vmt_poly_x2pow     out[i] = x^(2^(q_lo + i)) mod mu for q_lo <= q <= q_hi,
 *                      nw words per entry
 */
int vmt_poly_minpoly(const uint64_t* bits, int64_t n, uint64_t* mu_out, int64_t cap_words);
int vmt_poly_mulmod(const uint64_t* a, const uint64_t* b, const uint64_t* mu, uint64_t* out, int64_t nw);
int vmt_poly_x2pow(const uint64_t* mu, int64_t nw, int q_lo, int q_hi, uint64_t* out);

/*
 * Twisted GFSR generators with run-time parameters (Sec. 2.1 eq. step with
 * other constants; Sec. 3.1 jump; the paper's future-work remark that the
 * construction applies to other F2-linear generators).  A state is n
 * uint32 words on the device, x_k .. x_{k+n-1} oldest first, each holding a
 * w-bit word.  The recurrence is
 *     x_{k+n} = x_{k+m} xor (y >> 1) xor (y odd ? a : 0),
 *     y = (upper w-r bits of x_k) | (lower r bits of x_{k+1}),
 * and an output is x_{k+n}, or with temper != 0 the tempering of eq.
 * (tempering) with shifts u, s, t, l and masks d, b, c, truncated to w bits.
 * Compiled state sizes: n = 4, 5 or 17 (VMT_EINVAL otherwise); 2 <= w <= 32,
 * 1 <= m < n, 1 <= r < w, a < 2^w.
 */
typedef struct vmt_tgfsr {
    int w, n, m, r;
    uint32_t a;
    int temper;
    int u, s, t, l;
    uint32_t d, b, c;
} vmt_tgfsr;
/*
 * vmt_tgfsr_jump -- replace each of `count` states (states: count x n words,
 * device) by c(F) X, c the polynomial of nbits bits in poly (host, bit i of
 * poly[i/64] = coefficient of x^i, copied before the call returns).  Runs the
 * window-correlation jump kernels of vmt_jump: kernel 0 one warp per state,
 * 1 one CTA per state.  With c = x^J mod the minimal polynomial of the
 * transition (vmt_poly_minpoly on output bits, then vmt_poly_x2pow /
 * vmt_poly_mulmod) this advances every state by J steps.  Allocates its
 * scratch from the stream-ordered pool.  Asynchronous on cuda_stream.
 */
int vmt_tgfsr_jump(const vmt_tgfsr* g, int64_t count, void* states, const uint64_t* poly, int64_t nbits, int kernel,
                   void* cuda_stream);
/*
 * vmt_tgfsr_generate -- `count` = G * lanes states advance n steps each;
 * output word k of lane t of group g is stored at out[(g * n + k) * lanes + t]
 * (device, uint32: the interleaved stream of eq. combseq for a V-generator
 * of `lanes` lanes), and the advanced states are written back, so calls
 * continue the streams.  Asynchronous on cuda_stream.
 */
int vmt_tgfsr_generate(const vmt_tgfsr* g, int64_t count, int lanes, void* states, int64_t n, void* out,
                       void* cuda_stream);

/*
 * vmt_jump_noalloc -- vmt_jump for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment variant of vmt_jump.
 *
 * vmt_jump allocates device scratch on every call (a polynomial row and a
 * table of lane-jump work items).  Some callers cannot do that: code running
 * while a framework's caching allocator holds all free HBM, latency-bound loops
 * that must not pay for cudaMalloc/cudaFree, or plug-ins whose host forbids
 * library allocations.  This entry point computes the same result as vmt_jump
 * (st, poly and nbits mean the same) but calls no cudaMalloc, cudaFree or other
 * allocating routine: its scratch is a static device array of about 515 KiB
 * inside libvmt.so, which every GPU that loads the library keeps until the
 * process exits.
 *   - count * lanes of st must not exceed VMT_NOALLOC_MAX_LANE_STATES; larger
 *     states are rejected with VMT_EINVAL (nothing is enqueued);
 *   - the first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it with the
 *     id of the device's CUDA context; make that first call before any stream
 *     capture.  A call in a new context of the device (after cudaDeviceReset)
 *     looks the address up again;
 *   - all calls share the one array, which keeps the previous call's
 *     contents: each call rewrites the polynomial row and the work items it
 *     uses; calls whose work overlaps on the GPU (different streams without
 *     ordering) race on it, so order them on one stream or with events;
 *   - poly is read before the call returns, from any kind of host memory
 *     (pageable or pinned): its words travel to the GPU as a kernel parameter,
 *     so the call issues no copy and never waits for `cuda_stream`.
 */
#define VMT_NOALLOC_MAX_LANE_STATES 16384
int vmt_jump_noalloc(vmt_state* st, const uint64_t* poly, int64_t nbits, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VMT_H */
