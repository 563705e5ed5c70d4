// serve.cu -- request server for V-family generation (continuous batching).
//
// A request asks for n outputs of one fresh V-generator (variant, lanes M,
// seed, jump offset d; Sec. 3 and 3.1).  The server keeps a FIFO of submitted
// requests and a worker thread that, as long as memory allows, admits the
// queue head into the next batch: its generator state (M * n_units words)
// counts against the state budget until the batch has finished, its output
// against the output budget until the client releases it.  A batch groups its
// requests by kernel (variant, M, output type); per group one batched
// initialisation (seeding, per-request jump offsets, lane de-phasing) runs on
// the init stream and one persistent ragged generation (requests longest
// first) on the generation stream, after the group's init.  Batches are
// launched as soon as requests are admitted, so the initialisation of a new
// batch (ALU-bound jumps) overlaps the generation of the previous one
// (HBM-bound stores).  Completion is signalled from the stream by a host
// function that stamps the requests' completion times.
//
// Requests of at most kExpressOutputs outputs may also go ahead of the queue
// in batches of their own on express slots, one per variant, whose streams
// have the highest priority: their latency is then a few short launches, not
// the queue plus a batch of long requests, and a small MT19937 request never
// waits for an SFMT19937 jump chain.  Their outputs count
// against an express budget (a sixteenth of the output budget), so they never
// take output memory that a waiting request needs; they pass others only where
// the first request they pass still fits the state budget afterwards.
//
// Failure handling, all on the host: a request that can never fit the budgets
// or has invalid parameters fails alone (status < 0) and the server goes on;
// vmt_server_wait gives up after its timeout with VMT_ETIMEOUT; destroying the
// server waits for the batches in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "vmt_internal.hpp"

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int words_per_out(int variant, int dtype)
{
    if (variant == VMT_MT19937_64) return 1;
    return (dtype == VMT_U64 || dtype == VMT_F64) ? 2 : 1;
}

int out_bytes(int dtype) { return (dtype == VMT_U32 || dtype == VMT_F32) ? 4 : 8; }

// chunks of a request of w native words (the last one takes the rest)
int64_t n_chunks(int variant, int lanes, int64_t w)
{
    const int64_t C = vmt::chunk_words(variant, lanes);
    return std::min<int64_t>((w + C - 1) / C, vmt::kChunkRows + 1);
}

constexpr int kRegular = 4;                 // slots for batches of any request
constexpr int kSlots = kRegular + 3;        // + one express slot per variant (small requests only)
inline bool is_express(int slot) { return slot >= kRegular; }
inline int express_slot(int variant) { return kRegular + variant; }
constexpr int64_t kExpressOutputs = 16384;   // "small": at most this many outputs
constexpr size_t kExpressScan = 4096;        // queue entries an admission pass looks at
constexpr bool kSmallWaitsForExpress = true; // small requests run only in express batches
constexpr int kMaxGroups = 16;     // kernels per batch
constexpr int kMaxUnits = 65536;   // units (requests or chunks of requests) per batch

struct Req {
    vmt_request r{};
    int status = VMT_SERVER_QUEUED;
    void* out = nullptr;
    int64_t bytes = 0;
    int64_t state_bytes = 0;
    int64_t chunks = 1;      // generators it runs on (one per chunk)
    int launch_rc = VMT_OK;  // set when its own launch step failed (it fails alone)
    bool admitted = false;   // its output bytes count against the budget
    bool express = false;    // ... against the express budget
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Slot {
    cudaStream_t s_init[3] = {}, s_gen = nullptr;   // this slot's batches run here (init: one per variant)
    cudaEvent_t ev_init[3] = {};                    // end of a variant's initialisation
    vmt::UnitDesc* h_units = nullptr;
    vmt::UnitDesc* d_units = nullptr;
    int* d_counter = nullptr;
    uint64_t* h_seeds = nullptr;
    uint64_t* h_jumps = nullptr;
    int2* h_map = nullptr;    // (request, chunk) of every chunk state
    int2* d_map = nullptr;
    cudaEvent_t ev[3] = {};   // batch start, end of initialisation, end of generation
    bool busy = false;
};

struct Batch;
struct HostDone {
    vmt_server* srv;
    Batch* b;
};

struct Batch {
    int slot = -1;
    std::vector<uint64_t> ids;
    std::vector<vmt_state*> states;
    int64_t state_bytes = 0;
    int rc = VMT_OK;                     // launch error, given to its requests at retirement
    std::atomic<bool> gpu_done{false};   // set by the stream's host function
    double t_done = 0;
    HostDone cb;
};

}  // namespace

struct vmt_server {
    vmt_server_config cfg{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> queue;
    std::deque<uint64_t> done_q;   // requests that reached a final status, in that order
    std::unordered_map<uint64_t, Req> reqs;
    std::deque<Batch*> inflight;
    Slot slots[kSlots];
    int64_t used_state = 0, used_out = 0, peak_state = 0, peak_out = 0;
    int64_t used_out_express = 0;   // outputs of express requests (budget: output budget / 16)
    int64_t batches = 0, completed = 0, failed = 0, bytes_out = 0;
    double host_launch_s = 0, init_gpu_s = 0, batch_gpu_s = 0;
    int64_t cancelled = 0;
    int64_t express_batches = 0, express_completed = 0;
    double queued_s = 0, running_s = 0, express_queued_s = 0, express_running_s = 0;
    double express_init_gpu_s = 0, express_batch_gpu_s = 0;
    std::atomic<int> inject_alloc{0};   // output allocations still to fail (fault injection)
    cudaMemPool_t pool = nullptr;   // states and outputs
    // Memory is freed on a stream of its own, only ever after the kernels that
    // used it have finished, so reuse of a freed block never waits for other work.
    cudaStream_t s_free = nullptr;
    uint64_t next_id = 1;
    bool stop = false;
    int device = 0;
    std::thread worker;
};

namespace {

// Runs on the CUDA runtime's callback thread once the batch's work is done.  It
// takes no lock and makes no CUDA call: it stamps the time and raises a flag
// that the worker picks up.
void CUDART_CB on_batch_done(void* p)
{
    HostDone* h = static_cast<HostDone*>(p);
    vmt_server* srv = h->srv;   // read before the flag: the worker may free the batch right after it
    h->b->t_done = now_s();
    h->b->gpu_done.store(true, std::memory_order_release);
    srv->cv_work.notify_all();
}

// Launch one batch.  Per variant, on that variant's init stream of the slot
// (the three variants initialise concurrently): one batched initialisation
// of all its requests' generators (seeding and jump offsets once, the lane
// fan-out per kernel group (lanes, output type)); requests longer than one
// chunk (vmt::chunk_words) are cut at chunk boundaries, chunk c >= 1 getting
// its own generator, the request's lanes advanced to S word c * chunk (one
// device-side jump per lane).  Then per kernel group one persistent ragged
// launch over all chunks, longest first, on the slot's generation stream,
// after its variant's initialisation.
int launch_batch(vmt_server* s, Batch* b, std::vector<Req*>& rq)
{
    Slot& sl = s->slots[b->slot];
    cudaStream_t s_gen = sl.s_gen;
    cudaEventRecord(sl.ev[0], s_gen);
    // variant -> kernel group (lanes, dtype) -> request indices
    std::map<int, std::map<std::pair<int, int>, std::vector<size_t>>> by_variant;
    for (size_t i = 0; i < rq.size(); ++i)
        by_variant[rq[i]->r.variant][{rq[i]->r.lanes, rq[i]->r.dtype}].push_back(i);
    int64_t seed0 = 0, unit0 = 0, map0 = 0;
    int gk = 0;
    int rc = VMT_OK;
    for (auto& vv : by_variant) {
        const int variant = vv.first;
        cudaStream_t s_init = sl.s_init[variant];
        cudaStreamWaitEvent(s_init, sl.ev[0], 0);
        // one initialisation for the variant, one state object per group
        std::vector<int> lanes_of;
        std::vector<int64_t> counts;
        int64_t k_all = 0;
        for (auto& kv : vv.second) {
            lanes_of.push_back(kv.first.first);
            counts.push_back(static_cast<int64_t>(kv.second.size()));
            for (size_t i : kv.second) {
                sl.h_seeds[seed0 + k_all] = rq[i]->r.seed;
                sl.h_jumps[seed0 + k_all] = rq[i]->r.jump;
                ++k_all;
            }
        }
        const int nsub = static_cast<int>(counts.size());
        std::vector<vmt_state*> sts(static_cast<size_t>(nsub), nullptr);
        rc = vmt::init_multi_impl(sts.data(), variant, nsub, lanes_of.data(), counts.data(), sl.h_seeds + seed0,
                                  sl.h_jumps + seed0, s_init, true, s->pool, vmt::kJumpShared);
        if (rc) return rc;
        for (vmt_state* st : sts) b->states.push_back(st);
        seed0 += k_all;
        // per group: outputs, chunk generators and their jumps
        std::vector<vmt_state*> csts(static_cast<size_t>(nsub), nullptr);
        int gi = 0;
        for (auto& kv : vv.second) {
            const int lanes = kv.first.first, dtype = kv.first.second;
            const auto& idx = kv.second;
            const int64_t k = static_cast<int64_t>(idx.size());
            const int wpo = words_per_out(variant, dtype);
            for (int64_t i = 0; i < k; ++i) {
                Req* q = rq[idx[static_cast<size_t>(i)]];
                // an injected failure stands for a failed allocation call
                int inj = s->inject_alloc.load();
                while (inj > 0 && !s->inject_alloc.compare_exchange_weak(inj, inj - 1)) {
                }
                if (inj > 0 || cudaMallocFromPoolAsync(&q->out, static_cast<size_t>(std::max<int64_t>(q->bytes, 16)),
                                                       s->pool, s_init) != cudaSuccess) {
                    if (inj <= 0) cudaGetLastError();
                    q->out = nullptr;
                    q->launch_rc = VMT_ENOMEM;   // this request fails alone
                }
            }
            // chunks: request i, chunk c in 1..P_i-1
            int64_t nchunk = 0;
            for (int64_t i = 0; i < k; ++i) {
                if (!rq[idx[static_cast<size_t>(i)]]->out) continue;
                const int64_t P = n_chunks(variant, lanes, rq[idx[static_cast<size_t>(i)]]->r.n * wpo);
                for (int64_t c = 1; c < P; ++c)
                    sl.h_map[map0 + nchunk++] = make_int2(static_cast<int>(i), static_cast<int>(c));
            }
            if (nchunk) {
                rc = vmt::alloc_states_async(&csts[static_cast<size_t>(gi)], variant, lanes, nchunk, s_init, s->pool);
                if (rc) return rc;
                b->states.push_back(csts[static_cast<size_t>(gi)]);
                cudaMemcpyAsync(sl.d_map + map0, sl.h_map + map0, static_cast<size_t>(nchunk) * sizeof(int2),
                                cudaMemcpyHostToDevice, s_init);
                rc = vmt::launch_chunk_jumps(sts[static_cast<size_t>(gi)], csts[static_cast<size_t>(gi)],
                                             sl.d_map + map0, s_init, vmt::kJumpShared);
                if (rc) return rc;
            }
            map0 += nchunk;
            ++gi;
        }
        cudaEventRecord(sl.ev_init[variant], s_init);
        cudaStreamWaitEvent(s_gen, sl.ev_init[variant], 0);
        // generation per group: chunk 0 of every request on its own generator,
        // chunks >= 1 on the chunk generators; the last chunk takes the rest
        gi = 0;
        for (auto& kv : vv.second) {
            const int lanes = kv.first.first, dtype = kv.first.second;
            const auto& idx = kv.second;
            const int64_t k = static_cast<int64_t>(idx.size());
            const int wpo = words_per_out(variant, dtype);
            const int64_t gen_bytes = vmt::state_bytes_per_gen(variant, lanes);
            const int eb = out_bytes(dtype);
            const vmt_state* st = sts[static_cast<size_t>(gi)];
            const vmt_state* cst = csts[static_cast<size_t>(gi)];
            std::vector<vmt::UnitDesc> units;
            int64_t ck = 0;
            for (int64_t i = 0; i < k; ++i) {
                Req* q = rq[idx[static_cast<size_t>(i)]];
                const int64_t w = q->r.n * wpo;
                if (w == 0 || !q->out) continue;
                const int64_t C = vmt::chunk_words(variant, lanes);
                const int64_t P = n_chunks(variant, lanes, w);
                for (int64_t c = 0; c < P; ++c) {
                    vmt::UnitDesc u{};
                    const int64_t w0 = c * C, w1 = (c == P - 1) ? w : (c + 1) * C;
                    if (c == 0) {
                        u.state = static_cast<char*>(st->d_states) + i * gen_bytes;
                        u.pos = st->d_pos + i;
                    } else {
                        u.state = static_cast<char*>(cst->d_states) + ck * gen_bytes;
                        u.pos = cst->d_pos + ck;
                        ++ck;
                    }
                    u.total = w1 - w0;
                    u.out = static_cast<char*>(q->out) + (w0 / wpo) * eb;
                    units.push_back(u);
                }
            }
            std::stable_sort(units.begin(), units.end(),
                             [](const vmt::UnitDesc& x, const vmt::UnitDesc& y) { return x.total > y.total; });
            const int64_t nu = static_cast<int64_t>(units.size());
            if (nu) {
                std::memcpy(sl.h_units + unit0, units.data(), static_cast<size_t>(nu) * sizeof(vmt::UnitDesc));
                cudaMemcpyAsync(sl.d_units + unit0, sl.h_units + unit0,
                                static_cast<size_t>(nu) * sizeof(vmt::UnitDesc), cudaMemcpyHostToDevice, s_gen);
                rc = vmt::launch_unit_table(variant, lanes, dtype, sl.d_units + unit0, nu, sl.d_counter + gk, s_gen,
                                            true);
                if (rc) return rc;
            }
            unit0 += nu;
            ++gk;
            ++gi;
        }
    }
    return VMT_OK;
}

// Finished batches leave the in-flight list; returns their states, to be
// released after the lock is dropped (no CUDA call is made under the lock).
std::vector<std::pair<vmt_state*, cudaStream_t>> retire(vmt_server* s, std::vector<int>& slots)   // with s->mu held
{
    std::vector<std::pair<vmt_state*, cudaStream_t>> to_free;
    for (size_t i = 0; i < s->inflight.size();) {
        Batch* b = s->inflight[i];
        if (!b->gpu_done.load(std::memory_order_acquire)) {
            ++i;
            continue;
        }
        s->inflight.erase(s->inflight.begin() + static_cast<std::ptrdiff_t>(i));
        for (vmt_state* st : b->states) to_free.push_back({st, s->s_free});
        s->used_state -= b->state_bytes;
        for (uint64_t id : b->ids) {
            auto it = s->reqs.find(id);
            if (it == s->reqs.end()) continue;
            if (it->second.status == VMT_SERVER_RUNNING && (b->rc || it->second.launch_rc)) {
                // reported only now: its batch's kernels have finished
                it->second.status = b->rc ? b->rc : it->second.launch_rc;
                ++s->failed;
                s->done_q.push_back(id);
            } else if (it->second.status == VMT_SERVER_RUNNING) {
                Req& q = it->second;
                q.status = VMT_SERVER_DONE;
                q.t_done = b->t_done;
                (q.express ? s->express_queued_s : s->queued_s) += q.t_admit - q.t_submit;
                (q.express ? s->express_running_s : s->running_s) += q.t_done - q.t_admit;
                if (q.express) ++s->express_completed;
                ++s->completed;
                s->bytes_out += it->second.bytes;
                s->done_q.push_back(id);
            }
        }
        slots.push_back(b->slot);   // its events are read before the slot is reused
        delete b;
        s->cv_done.notify_all();
    }
    return to_free;
}

void worker_main(vmt_server* s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        std::vector<int> done_slots;
        const auto to_free = retire(s, done_slots);
        if (!done_slots.empty()) {
            lk.unlock();
            for (const auto& f : to_free) vmt::free_state_async(f.first, f.second);
            float t_init = 0, t_all = 0, x_init = 0, x_all = 0, ms = 0;
            for (int i : done_slots) {
                const bool x = is_express(i);
                if (cudaEventElapsedTime(&ms, s->slots[i].ev[0], s->slots[i].ev[1]) == cudaSuccess)
                    (x ? x_init : t_init) += ms;
                if (cudaEventElapsedTime(&ms, s->slots[i].ev[0], s->slots[i].ev[2]) == cudaSuccess)
                    (x ? x_all : t_all) += ms;
            }
            cudaGetLastError();
            lk.lock();
            s->init_gpu_s += 1e-3 * (t_init + x_init);
            s->batch_gpu_s += 1e-3 * (t_all + x_all);
            s->express_init_gpu_s += 1e-3 * x_init;
            s->express_batch_gpu_s += 1e-3 * x_all;
            for (int i : done_slots) s->slots[i].busy = false;
        }
        if (s->stop && s->queue.empty() && s->inflight.empty()) break;
        std::vector<Req*> rq;
        std::vector<uint64_t> ids;
        std::map<std::tuple<int, int, int>, int> kinds;
        int64_t add_state = 0, units = 0;
        // false when the request would exceed a batch limit (kernel groups, units)
        auto fits_batch = [&](const Req& q) {
            const auto key = std::make_tuple(q.r.variant, q.r.lanes, q.r.dtype);
            if (!kinds.count(key) && static_cast<int>(kinds.size()) == kMaxGroups) return false;
            return units + q.chunks <= kMaxUnits;
        };
        auto admit = [&](Req& q, uint64_t id, bool express) {
            units += q.chunks;
            kinds[std::make_tuple(q.r.variant, q.r.lanes, q.r.dtype)] = 1;
            add_state += q.state_bytes;
            (express ? s->used_out_express : s->used_out) += q.bytes;
            q.admitted = true;
            q.express = express;
            q.t_admit = now_s();
            q.status = VMT_SERVER_RUNNING;
            rq.push_back(&q);
            ids.push_back(id);
        };
        int slot = -1;
        for (int v = VMT_MT19937_32; v <= VMT_SFMT19937 && slot < 0; ++v) {
            if (s->slots[express_slot(v)].busy) continue;
            // express batch of variant v: its small requests go ahead of the
            // queue on a slot of their own, so that they never wait behind
            // long ones nor behind another variant's jumps.  Their outputs
            // count against an express budget of their own; the first queued
            // request they pass keeps its claim on the state budget: a small
            // request goes ahead only if that one would still fit after it.
            const int64_t express_budget = s->cfg.output_budget_bytes / 16;
            int64_t claim_state = 0;
            bool claimed = false;
            for (size_t k = 0; k < s->queue.size() && k < kExpressScan &&
                               static_cast<int>(rq.size()) < s->cfg.max_batch;) {
                const uint64_t id = s->queue[k];
                Req& q = s->reqs[id];
                const bool never = q.state_bytes > s->cfg.state_budget_bytes || q.bytes > s->cfg.output_budget_bytes;
                if (never || q.r.n > kExpressOutputs || q.bytes > express_budget) {
                    if (!never && !claimed) {
                        claimed = true;
                        claim_state = q.state_bytes;
                    }
                    ++k;
                    continue;
                }
                if (q.r.variant != v) {
                    ++k;
                    continue;
                }
                if (s->used_state + add_state + q.state_bytes + claim_state > s->cfg.state_budget_bytes ||
                    s->used_out_express + q.bytes > express_budget || !fits_batch(q))
                    break;
                admit(q, id, true);
                s->queue.erase(s->queue.begin() + static_cast<std::ptrdiff_t>(k));
            }
            if (!rq.empty()) slot = express_slot(v);
        }
        if (slot < 0)
            for (int i = 0; i < kRegular; ++i)
                if (!s->slots[i].busy) {
                    slot = i;
                    break;
                }
        // admission: FIFO, as long as both budgets hold; small requests that
        // the express budget can hold are left to the express slots (a
        // regular batch would make them wait for its longest request)
        for (size_t k = 0; slot >= 0 && !is_express(slot) && k < s->queue.size() && k < kExpressScan &&
                           static_cast<int>(rq.size()) < s->cfg.max_batch;) {
            const uint64_t id = s->queue[k];
            Req& q = s->reqs[id];
            if (q.state_bytes > s->cfg.state_budget_bytes || q.bytes > s->cfg.output_budget_bytes) {
                q.status = VMT_ENOMEM;   // can never be admitted
                ++s->failed;
                s->done_q.push_back(id);
                s->queue.erase(s->queue.begin() + static_cast<std::ptrdiff_t>(k));
                s->cv_done.notify_all();
                continue;
            }
            if (kSmallWaitsForExpress && q.r.n <= kExpressOutputs && q.bytes <= s->cfg.output_budget_bytes / 16) {
                ++k;
                continue;
            }
            if (s->used_state + add_state + q.state_bytes > s->cfg.state_budget_bytes ||
                s->used_out + q.bytes > s->cfg.output_budget_bytes || !fits_batch(q))
                break;
            admit(q, id, false);
            s->queue.erase(s->queue.begin() + static_cast<std::ptrdiff_t>(k));
        }
        if (rq.empty()) {
            // nothing to launch: sleep until a submit, a release or a finished
            // batch (the lock is released while waiting)
            s->cv_work.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        s->used_state += add_state;
        s->peak_state = std::max(s->peak_state, s->used_state);
        s->peak_out = std::max(s->peak_out, s->used_out + s->used_out_express);
        Batch* b = new Batch();
        b->slot = slot;
        b->ids = ids;
        b->state_bytes = add_state;
        b->cb = HostDone{s, b};
        s->slots[slot].busy = true;
        ++s->batches;
        if (is_express(slot)) ++s->express_batches;
        lk.unlock();
        const double t0 = now_s();
        const int rc = launch_batch(s, b, rq);
        // end of initialisation: all variants' init streams joined into the first
        Slot& sl = s->slots[slot];
        cudaStreamWaitEvent(sl.s_init[0], sl.ev_init[1], 0);
        cudaStreamWaitEvent(sl.s_init[0], sl.ev_init[2], 0);
        cudaEventRecord(sl.ev[1], sl.s_init[0]);
        cudaEventRecord(s->slots[slot].ev[2], s->slots[slot].s_gen);
        cudaLaunchHostFunc(s->slots[slot].s_gen, on_batch_done, &b->cb);
        const double t1 = now_s();
        lk.lock();
        s->host_launch_s += t1 - t0;
        b->rc = rc;
        s->inflight.push_back(b);
    }
}

}  // namespace

namespace {
bool valid_request(const vmt_request* r)
{
    const bool lanes_ok = r->lanes == 1 || r->lanes == 2 || r->lanes == 4 || r->lanes == 8 || r->lanes == 16;
    return !(r->variant < 0 || r->variant > 2 || !lanes_ok || r->dtype < VMT_U32 || r->dtype > VMT_F64 || r->n < 0 ||
             (r->variant == VMT_MT19937_64 && r->dtype == VMT_U32) ||
             r->n * words_per_out(r->variant, r->dtype) > (int64_t(1) << 30) ||
             (words_per_out(r->variant, r->dtype) == 2 && r->lanes < 2));
}

Req make_req(const vmt_request* r, double t)
{
    Req q;
    q.r = *r;
    q.bytes = r->n * out_bytes(r->dtype);
    q.chunks = std::max<int64_t>(n_chunks(r->variant, r->lanes, r->n * words_per_out(r->variant, r->dtype)), 1);
    q.state_bytes = q.chunks * (vmt::state_bytes_per_gen(r->variant, r->lanes) + 64);
    q.t_submit = t;
    return q;
}
}  // namespace

extern "C" {

int vmt_server_create(vmt_server** out, const vmt_server_config* cfg)
{
    if (!out || !cfg) {
        vmt::set_last_error("vmt_server_create: null argument");
        return VMT_EINVAL;
    }
    if (cfg->max_batch < 1 || cfg->max_batch > 4096 || cfg->state_budget_bytes <= 0 || cfg->output_budget_bytes <= 0) {
        vmt::set_last_error("vmt_server_create: max_batch must be in 1..4096 and budgets positive");
        return VMT_EINVAL;
    }
    vmt_server* s = new vmt_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->device);
    // the server's pool keeps up to both budgets' bytes mapped between requests
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    bool ok = cudaMemPoolCreate(&s->pool, &props) == cudaSuccess;
    if (ok) {
        uint64_t keep = static_cast<uint64_t>(cfg->state_budget_bytes) + static_cast<uint64_t>(cfg->output_budget_bytes);
        // A block freed on one stream is never handed to an allocation on
        // another by making the second stream wait for the first: the init
        // streams free their scratch at the end of long jump chains, and an
        // express batch must not queue behind a regular batch's chain for
        // its memory.  Blocks whose frees have completed are still reused.
        int no_wait = 0;
        ok = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess &&
             cudaMemPoolSetAttribute(s->pool, cudaMemPoolReuseAllowInternalDependencies, &no_wait) == cudaSuccess &&
             cudaStreamCreateWithFlags(&s->s_free, cudaStreamNonBlocking) == cudaSuccess;
    }
    // three priorities: the express slot's work above the regular slots'
    // initialisation (short jump launches), above the regular generation
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    const int prio_init = prio_hi < prio_lo ? prio_hi + 1 : prio_hi;   // greater priority = smaller number
    for (int i = 0; i < kSlots && ok; ++i) {
        Slot& sl = s->slots[i];
        const size_t n = static_cast<size_t>(cfg->max_batch);
        const size_t nu = static_cast<size_t>(kMaxUnits);
        // initialisation (short jump launches) is scheduled ahead of generation
        // blocks still waiting for an SM (every generation unit has its own
        // CTA, so an SM frees up whenever one finishes); the express slot's
        // initialisation and generation go ahead of both
        ok = cudaStreamCreateWithPriority(&sl.s_gen, cudaStreamNonBlocking, is_express(i) ? prio_hi : prio_lo) ==
                 cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void**>(&sl.h_units), nu * sizeof(vmt::UnitDesc), 0) == cudaSuccess &&
             cudaMalloc(reinterpret_cast<void**>(&sl.d_units), nu * sizeof(vmt::UnitDesc)) == cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void**>(&sl.h_map), nu * sizeof(int2), 0) == cudaSuccess &&
             cudaMalloc(reinterpret_cast<void**>(&sl.d_map), nu * sizeof(int2)) == cudaSuccess &&
             cudaMalloc(reinterpret_cast<void**>(&sl.d_counter), kMaxGroups * sizeof(int)) == cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void**>(&sl.h_seeds), n * 8, 0) == cudaSuccess &&
             cudaHostAlloc(reinterpret_cast<void**>(&sl.h_jumps), n * 8, 0) == cudaSuccess;
        for (int e = 0; e < 3 && ok; ++e)
            ok = cudaEventCreate(&sl.ev[e]) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev_init[e], cudaEventDisableTiming) == cudaSuccess &&
                 cudaStreamCreateWithPriority(&sl.s_init[e], cudaStreamNonBlocking,
                                              is_express(i) ? prio_hi : prio_init) == cudaSuccess;
    }
    if (ok && cfg->reserve) {
        // map the budgets now: one allocation of their sum, freed back to the pool
        void* p = nullptr;
        const size_t bytes = static_cast<size_t>(cfg->state_budget_bytes) + static_cast<size_t>(cfg->output_budget_bytes);
        if (cudaMallocFromPoolAsync(&p, bytes, s->pool, s->slots[0].s_gen) != cudaSuccess) {
            cudaGetLastError();
            vmt::set_last_error("vmt_server_create: the budgets do not fit in device memory");
            vmt_server_destroy(s);
            return VMT_ENOMEM;
        }
        ok = cudaFreeAsync(p, s->slots[0].s_gen) == cudaSuccess &&
             cudaStreamSynchronize(s->slots[0].s_gen) == cudaSuccess;
        for (int v = VMT_MT19937_32; v <= VMT_SFMT19937 && ok; ++v) {
            const int rc = vmt_prepare(v, s->slots[0].s_gen);
            if (rc) {
                vmt_server_destroy(s);
                return rc;
            }
        }
    }
    if (!ok) {
        vmt::set_last_error("vmt_server_create: CUDA resources could not be created");
        vmt_server_destroy(s);
        return VMT_ECUDA;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return VMT_OK;
}


int vmt_server_submit(vmt_server* s, const vmt_request* r, uint64_t* id)
{
    if (!s || !r || !id) {
        vmt::set_last_error("vmt_server_submit: null argument");
        return VMT_EINVAL;
    }
    return vmt_server_submit_many(s, r, 1, id);
}

int vmt_server_submit_many(vmt_server* s, const vmt_request* reqs, int64_t n, uint64_t* ids)
{
    if (!s || n < 0 || (n > 0 && (!reqs || !ids))) {
        vmt::set_last_error("vmt_server_submit: null argument");
        return VMT_EINVAL;
    }
    for (int64_t i = 0; i < n; ++i)
        if (!valid_request(&reqs[i])) {
            vmt::set_last_error("vmt_server_submit: invalid request");
            return VMT_EINVAL;
        }
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int64_t i = 0; i < n; ++i) {
            ids[i] = s->next_id++;
            s->reqs.emplace(ids[i], make_req(&reqs[i], t));
            s->queue.push_back(ids[i]);
        }
    }
    s->cv_work.notify_all();
    return VMT_OK;
}

int vmt_server_poll(vmt_server* s, uint64_t id, int* status, void** out_dev, int64_t* bytes, double* latency_s)
{
    if (!s) return VMT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        vmt::set_last_error("vmt_server_poll: unknown request id");
        return VMT_EINVAL;
    }
    const Req& q = it->second;
    if (status) *status = q.status;
    if (out_dev) *out_dev = q.status == VMT_SERVER_DONE ? q.out : nullptr;
    if (bytes) *bytes = q.bytes;
    if (latency_s) *latency_s = q.status == VMT_SERVER_DONE ? q.t_done - q.t_submit : -1.0;
    return VMT_OK;
}

int vmt_server_wait(vmt_server* s, uint64_t id, int timeout_ms)
{
    if (!s) return VMT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto it = s->reqs.find(id);
        return it == s->reqs.end() || it->second.status == VMT_SERVER_DONE || it->second.status < 0;
    });
    if (!ok) {
        vmt::set_last_error("vmt_server_wait: timed out");
        return VMT_ETIMEOUT;
    }
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return VMT_EINVAL;
    return it->second.status < 0 ? it->second.status : VMT_OK;
}

int vmt_server_copy(vmt_server* s, uint64_t id, void* host_buf, int64_t cap)
{
    void* out = nullptr;
    int64_t bytes = 0;
    int status = 0;
    const int rc = vmt_server_poll(s, id, &status, &out, &bytes, nullptr);
    if (rc) return rc;
    if (status != VMT_SERVER_DONE) {
        vmt::set_last_error("vmt_server_copy: request not done");
        return VMT_EBUSY;
    }
    if (!host_buf || cap < bytes) {
        vmt::set_last_error("vmt_server_copy: host buffer too small");
        return VMT_EINVAL;
    }
    if (bytes && cudaMemcpy(host_buf, out, static_cast<size_t>(bytes), cudaMemcpyDeviceToHost) != cudaSuccess) {
        vmt::set_last_error("vmt_server_copy: copy failed");
        return VMT_ECUDA;
    }
    return VMT_OK;
}

int vmt_server_release(vmt_server* s, uint64_t id)
{
    if (!s) return VMT_EINVAL;
    void* out = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) {
            vmt::set_last_error("vmt_server_release: unknown request id");
            return VMT_EINVAL;
        }
        Req& q = it->second;
        if (q.status == VMT_SERVER_QUEUED || q.status == VMT_SERVER_RUNNING) {
            vmt::set_last_error("vmt_server_release: request still pending");
            return VMT_EBUSY;
        }
        out = q.out;
        if (q.admitted) (q.express ? s->used_out_express : s->used_out) -= q.bytes;
        s->reqs.erase(it);
    }
    if (out) cudaFreeAsync(out, s->s_free);
    s->cv_work.notify_all();
    return VMT_OK;
}

int vmt_server_next_done(vmt_server* s, int64_t timeout_us, uint64_t* id)
{
    if (!s || !id || timeout_us < 0) return VMT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    // ids of released requests are skipped (their owner has seen them already)
    auto ready = [&] {
        while (!s->done_q.empty() && !s->reqs.count(s->done_q.front())) s->done_q.pop_front();
        return !s->done_q.empty();
    };
    if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return VMT_ETIMEOUT;
    *id = s->done_q.front();
    s->done_q.pop_front();
    return VMT_OK;
}

int64_t vmt_server_next_done_many(vmt_server* s, int64_t timeout_us, uint64_t* ids, int* status, double* latency_s,
                                  int64_t cap)
{
    if (!s || timeout_us < 0 || cap < 0 || (cap > 0 && (!ids || !status || !latency_s))) return VMT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] {
        while (!s->done_q.empty() && !s->reqs.count(s->done_q.front())) s->done_q.pop_front();
        return !s->done_q.empty();
    };
    if (cap == 0 || !s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return 0;
    int64_t k = 0;
    while (k < cap && ready()) {
        const uint64_t id = s->done_q.front();
        s->done_q.pop_front();
        const Req& q = s->reqs[id];
        ids[k] = id;
        status[k] = q.status;
        latency_s[k] = q.status == VMT_SERVER_DONE ? q.t_done - q.t_submit : -1.0;
        ++k;
    }
    return k;
}

int vmt_server_release_many(vmt_server* s, const uint64_t* ids, int64_t n)
{
    if (!s || n < 0 || (n > 0 && !ids)) return VMT_EINVAL;
    int rc = VMT_OK;
    for (int64_t i = 0; i < n; ++i) {
        const int r = vmt_server_release(s, ids[i]);
        if (r != VMT_OK && rc == VMT_OK) rc = r;
    }
    return rc;
}

int vmt_server_cancel(vmt_server* s, uint64_t id)
{
    if (!s) return VMT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) {
        vmt::set_last_error("vmt_server_cancel: unknown request id");
        return VMT_EINVAL;
    }
    if (it->second.status != VMT_SERVER_QUEUED) {
        vmt::set_last_error("vmt_server_cancel: request already running or finished");
        return VMT_EBUSY;
    }
    auto q = std::find(s->queue.begin(), s->queue.end(), id);
    if (q != s->queue.end()) s->queue.erase(q);
    it->second.status = VMT_ECANCELED;
    ++s->cancelled;
    s->done_q.push_back(id);
    s->cv_done.notify_all();
    return VMT_OK;
}

int vmt_server_inject(vmt_server* s, int what, int count)
{
    if (!s || what != VMT_INJECT_ALLOC || count < 0) {
        vmt::set_last_error("vmt_server_inject: unknown fault or negative count");
        return VMT_EINVAL;
    }
    s->inject_alloc.store(count);
    return VMT_OK;
}

int vmt_server_stats(vmt_server* s, vmt_server_counters* out)
{
    if (!s || !out) return VMT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = static_cast<int64_t>(s->queue.size());
    out->in_flight_batches = static_cast<int64_t>(s->inflight.size());
    out->batches = s->batches;
    out->completed = s->completed;
    out->failed = s->failed;
    out->bytes_out = s->bytes_out;
    out->state_bytes_in_use = s->used_state;
    out->output_bytes_in_use = s->used_out + s->used_out_express;
    out->peak_state_bytes = s->peak_state;
    out->peak_output_bytes = s->peak_out;
    out->host_launch_s = s->host_launch_s;
    out->init_gpu_s = s->init_gpu_s;
    out->batch_gpu_s = s->batch_gpu_s;
    out->cancelled = s->cancelled;
    out->express_batches = s->express_batches;
    out->express_completed = s->express_completed;
    out->queued_s = s->queued_s;
    out->running_s = s->running_s;
    out->express_queued_s = s->express_queued_s;
    out->express_running_s = s->express_running_s;
    out->express_init_gpu_s = s->express_init_gpu_s;
    out->express_batch_gpu_s = s->express_batch_gpu_s;
    return VMT_OK;
}

void vmt_server_destroy(vmt_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& sl : s->slots) {
        if (sl.s_gen) cudaStreamSynchronize(sl.s_gen);
        for (cudaStream_t si : sl.s_init)
            if (si) cudaStreamSynchronize(si);
    }
    for (auto& kv : s->reqs)
        if (kv.second.out) cudaFreeAsync(kv.second.out, s->s_free);
    if (s->s_free) cudaStreamSynchronize(s->s_free);
    for (auto& sl : s->slots) {
        if (sl.s_gen) cudaStreamSynchronize(sl.s_gen);
        if (sl.h_units) cudaFreeHost(sl.h_units);
        if (sl.d_units) cudaFree(sl.d_units);
        if (sl.d_counter) cudaFree(sl.d_counter);
        if (sl.h_seeds) cudaFreeHost(sl.h_seeds);
        if (sl.h_jumps) cudaFreeHost(sl.h_jumps);
        if (sl.h_map) cudaFreeHost(sl.h_map);
        if (sl.d_map) cudaFree(sl.d_map);
        for (cudaEvent_t e : sl.ev)
            if (e) cudaEventDestroy(e);
        for (cudaStream_t si : sl.s_init)
            if (si) cudaStreamDestroy(si);
        for (cudaEvent_t e : sl.ev_init)
            if (e) cudaEventDestroy(e);
        if (sl.s_gen) cudaStreamDestroy(sl.s_gen);
    }
    if (s->s_free) cudaStreamDestroy(s->s_free);
    if (s->pool) cudaMemPoolDestroy(s->pool);   // its memory is returned once the frees above complete
    delete s;
}

}  // extern "C"
