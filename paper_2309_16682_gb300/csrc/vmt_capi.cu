// vmt_capi.cu -- the C ABI declared in include/vmt.h.
//
// Host-side orchestration only: argument checking, device memory, the jump
// polynomial tables and kernel launches.  Every step of the generator path
// (seeding, jump evaluation, twist, tempering, interleave, conversion, store)
// runs in the CUDA kernels of gen_mt.cu, gen_sfmt.cu and jump.cu; there is no
// host fallback for any of them.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "gf2poly.hpp"
#include "vmt_internal.hpp"

namespace vmt {
cudaError_t launch_generate_mt(int variant, int lanes, const GenArgs& a, cudaStream_t s);
cudaError_t launch_generate_sfmt(int lanes, const GenArgs& a, bool ragged, cudaStream_t s);
cudaError_t launch_convert(const void* words, long long words_per_gen, int word64, long long gens, long long wbeg,
                           int dtype, long long count, void* out, cudaStream_t s);

cudaError_t launch_generate(int variant, int lanes, const GenArgs& a, bool ragged, cudaStream_t s)
{
    if (variant == VMT_SFMT19937) return launch_generate_sfmt(lanes, a, ragged, s);
    return launch_generate_mt(variant, lanes, a, s);   // one CTA per generator: ragged needs nothing special
}
}  // namespace vmt

using vmt::gf2::Poly;

namespace {
thread_local std::string g_err;
}

void vmt::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

// ---------------------------------------------------------------------------
// tuning table: compiled kernel configuration per (variant, lanes), an index
// into that pair's rows of vmt::kKernelCfgs (0: the default)
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_lock;
int g_tune_kcfg[3][17] = {};
bool g_tune_env_read = false;

// candidate index of the phase-form kernel with `threads` threads (-1: none)
int phase_index(int variant, int lanes, int threads)
{
    const int n = vmt::kernel_cfg_count(variant, lanes);
    for (int i = 0; i < n; ++i) {
        const vmt::KernelCfg* c = vmt::kernel_cfg(variant, lanes, i);
        if (c->form == vmt::kPhase && c->threads == threads) return i;
    }
    return -1;
}

void read_tune_env_locked()
{
    if (g_tune_env_read) return;
    g_tune_env_read = true;
    // VMT_TUNE="mt32:16:1024,mt64:8:#2": a phase-form CTA size, or #index
    const char* e = std::getenv("VMT_TUNE");
    if (!e) return;
    std::string s(e);
    size_t i = 0;
    while (i < s.size()) {
        size_t j = s.find(',', i);
        if (j == std::string::npos) j = s.size();
        const std::string item = s.substr(i, j - i);
        int lanes = 0, val = 0;
        char name[8] = {0};
        bool by_index = false;
        bool ok = std::sscanf(item.c_str(), "%7[a-z0-9]:%d:#%d", name, &lanes, &val) == 3;
        if (ok) by_index = true;
        else ok = std::sscanf(item.c_str(), "%7[a-z0-9]:%d:%d", name, &lanes, &val) == 3;
        if (ok && lanes >= 0 && lanes <= 16) {
            const std::string n(name);
            const int v = n == "mt32" ? 0 : (n == "mt64" ? 1 : (n == "sfmt" ? 2 : -1));
            if (v >= 0) {
                const int idx = by_index ? val : phase_index(v, lanes, val);
                if (idx >= 0 && idx < vmt::kernel_cfg_count(v, lanes)) g_tune_kcfg[v][lanes] = idx;
            }
        }
        i = j + 1;
    }
}
}  // namespace

int vmt::tuned_kcfg(int variant, int lanes)
{
    if (variant < 0 || variant > 2 || lanes < 0 || lanes > 16) return 0;
    std::lock_guard<std::mutex> lk(g_tune_lock);
    read_tune_env_locked();
    return g_tune_kcfg[variant][lanes];
}

namespace {

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                                       \
    do {                                                                                                     \
        cudaError_t e_ = (expr);                                                                             \
        if (e_ != cudaSuccess) return fail(VMT_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool valid_variant(int v) { return v == VMT_MT19937_32 || v == VMT_MT19937_64 || v == VMT_SFMT19937; }
bool valid_lanes(int m) { return m == 1 || m == 2 || m == 4 || m == 8 || m == 16; }

// Lane spacing of Table "jvalues": J = 2^(19937 - log2 M).  Rows 0..15 of a
// variant's device table hold x^(s * 2^19933) mod mu, s = 0..15, so lane t of
// an M-lane generator uses row t * 16 / M.  Rows 16 .. 16+2040 hold the
// base-256 digit jumps x^(v * 256^i), i = 0..7, v = 1..255 (row 16 + 255 i + v - 1).
constexpr int kPeriodExp = 19937;
constexpr int kLaneRowQ = kPeriodExp - 4;   // J for M = 16
constexpr int kDigitRows = 8 * 255;
constexpr int kChunkRow0 = 16 + kDigitRows;   // first chunk row (chunk 1)
constexpr int kChainLo = 72;                // x^(2^q), q < 72, kept for d-jumps
constexpr int kChainHiFrom = kPeriodExp - 8;

struct VariantCtx {
    std::mutex mu_lock;
    bool ready = false;
    bool digits_ready = false;
    bool chunks_ready = false;
    std::unique_ptr<vmt::gf2::Modulus> mod;
    std::vector<Poly> chain_lo;    // q = 0 .. kChainLo-1
    std::vector<Poly> chain_hi;    // q = kChainHiFrom .. kPeriodExp
    std::vector<Poly> lane_rows;   // 16 rows
    int device = -1;
    uint32_t* d_table = nullptr;   // [16 + kDigitRows][kPolyWords]
    std::vector<int> row_deg;      // degree of each device row
    int* d_row_deg = nullptr;      // the same, on the device
};

VariantCtx g_ctx[3];
std::mutex g_cache_lock;
std::string g_cache_dir;

std::string cache_dir()
{
    std::lock_guard<std::mutex> lk(g_cache_lock);
    if (!g_cache_dir.empty()) return g_cache_dir;
    const char* e = std::getenv("VMT_CACHE_DIR");
    return e ? std::string(e) : std::string();
}

// -------------------------------------------------------------------------
// polynomial tables
// -------------------------------------------------------------------------
void to_rows(const Poly& p, uint32_t* row)
{
    std::memset(row, 0, sizeof(uint32_t) * vmt::kPolyWords);
    for (size_t w = 0; w < p.size() && 2 * w + 1 < static_cast<size_t>(vmt::kPolyWords); ++w) {
        row[2 * w] = static_cast<uint32_t>(p[w]);
        row[2 * w + 1] = static_cast<uint32_t>(p[w] >> 32);
    }
}

struct CacheHeader {
    char magic[8];
    int32_t version, variant, deg, nw, nlo, nhi;
};

bool load_cache(int variant, Poly& mu, std::vector<Poly>& lo, std::vector<Poly>& hi)
{
    const std::string dir = cache_dir();
    if (dir.empty()) return false;
    const std::string path = dir + "/minpoly_v" + std::to_string(variant) + ".bin";
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) return false;
    CacheHeader h{};
    bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && std::memcmp(h.magic, "VMTPOLY1", 8) == 0 && h.version == 1 &&
              h.variant == variant && h.nlo == kChainLo && h.nhi == kPeriodExp - kChainHiFrom + 1 && h.nw > 0 &&
              h.nw < 1024;
    if (ok) {
        mu.assign(static_cast<size_t>(h.nw) + 1, 0);
        ok = std::fread(mu.data(), 8, mu.size(), f) == mu.size();
        lo.assign(static_cast<size_t>(h.nlo), Poly(static_cast<size_t>(h.nw), 0));
        hi.assign(static_cast<size_t>(h.nhi), Poly(static_cast<size_t>(h.nw), 0));
        for (auto& p : lo) ok = ok && std::fread(p.data(), 8, p.size(), f) == p.size();
        for (auto& p : hi) ok = ok && std::fread(p.data(), 8, p.size(), f) == p.size();
        ok = ok && vmt::gf2::degree(mu) == h.deg;
    }
    std::fclose(f);
    return ok;
}

void save_cache(int variant, const Poly& mu, int nw, const std::vector<Poly>& lo, const std::vector<Poly>& hi)
{
    const std::string dir = cache_dir();
    if (dir.empty()) return;
    const std::string path = dir + "/minpoly_v" + std::to_string(variant) + ".bin";
    const std::string tmp = path + ".tmp" + std::to_string(reinterpret_cast<uintptr_t>(&lo));
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return;
    CacheHeader h{};
    std::memcpy(h.magic, "VMTPOLY1", 8);
    h.version = 1;
    h.variant = variant;
    h.deg = vmt::gf2::degree(mu);
    h.nw = nw;
    h.nlo = static_cast<int32_t>(lo.size());
    h.nhi = static_cast<int32_t>(hi.size());
    Poly m = mu;
    m.resize(static_cast<size_t>(nw) + 1, 0);
    bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(m.data(), 8, m.size(), f) == m.size();
    for (const auto& p : lo) ok = ok && std::fwrite(p.data(), 8, p.size(), f) == p.size();
    for (const auto& p : hi) ok = ok && std::fwrite(p.data(), 8, p.size(), f) == p.size();
    std::fclose(f);
    if (ok) std::rename(tmp.c_str(), path.c_str());
    else std::remove(tmp.c_str());
}

// Output bits of the variant's own generator, produced by the CUDA kernels
// (seed 5489, one lane): the sequence Berlekamp-Massey works on.
int sample_bits(int variant, int bit, int64_t nbits, std::vector<uint64_t>& packed, cudaStream_t st)
{
    const int n_units = vmt::units_per_lane(variant);
    const int wb = vmt::word_bytes(variant);
    const int64_t unit_bytes = static_cast<int64_t>(wb) * vmt::words_per_unit(variant);
    // words needed: one bit per native word (MT) or per element (SFMT)
    const int64_t words = (variant == VMT_SFMT19937) ? 4 * nbits : nbits;
    unsigned long long* d_seed = nullptr;
    void* d_state = nullptr;
    void* d_out = nullptr;
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_seed), 8, st));
    CUDA_TRY(cudaMallocAsync(&d_state, n_units * unit_bytes, st));
    CUDA_TRY(cudaMallocAsync(&d_out, words * wb, st));
    const unsigned long long seed = 5489ull;
    CUDA_TRY(cudaMemcpyAsync(d_seed, &seed, 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(vmt::launch_seed(variant, 1, d_seed, d_state, st));
    int* d_pos1 = nullptr;
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_pos1), sizeof(int), st));
    CUDA_TRY(vmt::launch_fill_int(d_pos1, 1, static_cast<int>(vmt::block_words(variant, 1)), st));
    vmt::GenArgs a{};
    a.states = d_state;
    a.gens = 1;
    a.gen0 = 0;
    a.pos = static_cast<int>(vmt::block_words(variant, 1));   // fresh state: the first output twists
    a.pos_dev = d_pos1;
    a.total = words;
    a.nseg = 1;
    a.seg[0].out = static_cast<char*>(d_out);
    a.seg[0].count = words;
    a.seg[0].wbeg = 0;
    a.seg[0].wend = words;
    a.seg[0].dtype = (variant == VMT_MT19937_64) ? VMT_U64 : VMT_U32;
    a.seg[0].fast = 0;
    CUDA_TRY(vmt::launch_generate(variant, 1, a, false, st));
    std::vector<unsigned char> host(static_cast<size_t>(words * wb));
    CUDA_TRY(cudaMemcpyAsync(host.data(), d_out, words * wb, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(d_seed, st);
    cudaFreeAsync(d_state, st);
    cudaFreeAsync(d_out, st);
    cudaFreeAsync(d_pos1, st);
    packed.assign(static_cast<size_t>((nbits + 63) / 64), 0);
    for (int64_t i = 0; i < nbits; ++i) {
        uint64_t v;
        if (variant == VMT_MT19937_64) std::memcpy(&v, &host[static_cast<size_t>(i) * 8], 8);
        else {
            uint32_t u;
            const int64_t widx = (variant == VMT_SFMT19937) ? 4 * i + bit / 32 : i;
            std::memcpy(&u, &host[static_cast<size_t>(widx) * 4], 4);
            v = u;
        }
        const int b = (variant == VMT_SFMT19937) ? bit % 32 : bit;
        if ((v >> b) & 1ull) packed[static_cast<size_t>(i >> 6)] |= 1ull << (i & 63);
    }
    return VMT_OK;
}

int ensure_variant(int variant, cudaStream_t st)
{
    VariantCtx& c = g_ctx[variant];
    std::lock_guard<std::mutex> lk(c.mu_lock);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (c.ready && c.device == dev) return VMT_OK;
    if (!c.ready) {
        Poly mu;
        std::vector<Poly> lo, hi;
        if (!load_cache(variant, mu, lo, hi)) {
            const int64_t nbits = 2 * 19968 + 256;
            std::vector<uint64_t> bits;
            const int top = (variant == VMT_MT19937_32) ? 31 : (variant == VMT_MT19937_64 ? 63 : 0);
            int rc = sample_bits(variant, top, nbits, bits, st);
            if (rc) return rc;
            mu = vmt::gf2::berlekamp_massey(bits.data(), nbits);
            if (variant == VMT_SFMT19937) {
                // the lcm over a few bit positions reaches the full minimal polynomial
                const int extra[] = {32, 64, 96, 1, 33, 65, 97};
                for (int b : extra) {
                    if (vmt::gf2::degree(mu) >= 19968) break;
                    rc = sample_bits(variant, b, nbits, bits, st);
                    if (rc) return rc;
                    Poly m2 = vmt::gf2::berlekamp_massey(bits.data(), nbits);
                    Poly g = vmt::gf2::gcd(mu, m2);
                    mu = vmt::gf2::mul_plain(mu, vmt::gf2::div_exact(m2, g));
                }
            }
            const int D = vmt::gf2::degree(mu);
            if ((variant != VMT_SFMT19937 && D != kPeriodExp) || (variant == VMT_SFMT19937 && D < kPeriodExp))
                return fail(VMT_ECUDA, "minimal polynomial has unexpected degree " + std::to_string(D));
            vmt::gf2::Modulus mod(mu);
            lo.clear();
            hi.clear();
            Poly r = mod.x_pow_2q(0);
            for (int q = 0; q <= kPeriodExp; ++q) {
                if (q < kChainLo) lo.push_back(r);
                if (q >= kChainHiFrom) hi.push_back(r);
                if (q < kPeriodExp) r = mod.sqr(r);
            }
            if (variant != VMT_SFMT19937) {
                // x^(2^p) = x mod mu for the primitive degree-p polynomial of MT
                Poly x(2, 0);
                x[0] = 2;
                if (vmt::gf2::degree(mod.reduce(x)) != 1 ||
                    !std::equal(hi.back().begin(), hi.back().end(), mod.reduce(x).begin()))
                    return fail(VMT_ECUDA, "minimal polynomial failed the x^(2^19937) = x check");
            }
            save_cache(variant, mu, mod.words(), lo, hi);
        }
        c.mod.reset(new vmt::gf2::Modulus(mu));
        c.chain_lo = std::move(lo);
        c.chain_hi = std::move(hi);
        // lane rows: x^(s * 2^19933), s = 0..15
        c.lane_rows.assign(16, Poly());
        Poly one(1, 1);
        c.lane_rows[0] = c.mod->reduce(one);
        const Poly& xJ = c.chain_hi[static_cast<size_t>(kLaneRowQ - kChainHiFrom)];
        for (int s = 1; s < 16; ++s) c.lane_rows[static_cast<size_t>(s)] = c.mod->mul(c.lane_rows[static_cast<size_t>(s - 1)], xJ);
        c.ready = true;
        c.digits_ready = false;
        c.device = -1;
    }
    if (c.device != dev) {
        const size_t rows = 16 + kDigitRows + vmt::kChunkRows;
        if (c.d_table) cudaFree(c.d_table);
        c.d_table = nullptr;
        CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&c.d_table), rows * vmt::kPolyWords * sizeof(uint32_t)));
        std::vector<uint32_t> host(16 * static_cast<size_t>(vmt::kPolyWords));
        c.row_deg.assign(rows, -1);
        for (int s = 0; s < 16; ++s) {
            to_rows(c.lane_rows[static_cast<size_t>(s)], &host[static_cast<size_t>(s) * vmt::kPolyWords]);
            c.row_deg[static_cast<size_t>(s)] = vmt::gf2::degree(c.lane_rows[static_cast<size_t>(s)]);
        }
        CUDA_TRY(cudaMemcpy(c.d_table, host.data(), host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
        if (c.d_row_deg) cudaFree(c.d_row_deg);
        c.d_row_deg = nullptr;
        CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(&c.d_row_deg), rows * sizeof(int)));
        CUDA_TRY(cudaMemcpy(c.d_row_deg, c.row_deg.data(), rows * sizeof(int), cudaMemcpyHostToDevice));
        c.device = dev;
        c.digits_ready = false;
        c.chunks_ready = false;
    }
    return VMT_OK;
}

// rows x^(c * kChunkBlocks * n) for chunks c = 1..kChunkRows
int ensure_chunks(int variant)
{
    VariantCtx& c = g_ctx[variant];
    std::lock_guard<std::mutex> lk(c.mu_lock);
    if (c.chunks_ready) return VMT_OK;
    const uint64_t delta = static_cast<uint64_t>(vmt::kChunkBlocks) * vmt::units_per_lane(variant);
    std::vector<uint32_t> host(static_cast<size_t>(vmt::kChunkRows) * vmt::kPolyWords);
    // rows 1..T serially, then T threads, thread i taking rows i, i + T, ...
    // (row j + T = row j * x^(T delta))
    constexpr int T = 16;
    std::vector<Poly> rows(static_cast<size_t>(vmt::kChunkRows) + 1);
    rows[1] = c.mod->x_pow(delta);
    for (int j = 2; j <= T; ++j) rows[static_cast<size_t>(j)] = c.mod->mul(rows[static_cast<size_t>(j - 1)], rows[1]);
    std::vector<std::thread> th;
    for (int i = 1; i <= T; ++i)
        th.emplace_back([&, i]() {
            for (int j = i + T; j <= vmt::kChunkRows; j += T)
                rows[static_cast<size_t>(j)] = c.mod->mul(rows[static_cast<size_t>(j - T)], rows[static_cast<size_t>(T)]);
        });
    for (auto& t : th) t.join();
    for (int j = 1; j <= vmt::kChunkRows; ++j) {
        to_rows(rows[static_cast<size_t>(j)], &host[static_cast<size_t>(j - 1) * vmt::kPolyWords]);
        c.row_deg[static_cast<size_t>(kChunkRow0 + j - 1)] = vmt::gf2::degree(rows[static_cast<size_t>(j)]);
    }
    CUDA_TRY(cudaMemcpy(c.d_table + static_cast<size_t>(kChunkRow0) * vmt::kPolyWords, host.data(),
                        host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c.d_row_deg, c.row_deg.data(), c.row_deg.size() * sizeof(int), cudaMemcpyHostToDevice));
    c.chunks_ready = true;
    return VMT_OK;
}

// base-256 digit rows for per-generator jump offsets d < 2^64
int ensure_digits(int variant)
{
    VariantCtx& c = g_ctx[variant];
    std::lock_guard<std::mutex> lk(c.mu_lock);
    if (c.digits_ready) return VMT_OK;
    std::vector<uint32_t> host(static_cast<size_t>(kDigitRows) * vmt::kPolyWords);
    std::vector<Poly> rows(static_cast<size_t>(kDigitRows));
    // x^(v 256^i) = (x^(256^i))^v; digit positions are independent -> threads
    std::vector<std::thread> th;
    for (int i = 0; i < 8; ++i)
        th.emplace_back([&, i]() {
            const Poly& base = c.chain_lo[static_cast<size_t>(8 * i)];
            Poly cur = base;
            for (int v = 1; v <= 255; ++v) {
                if (v > 1) cur = c.mod->mul(cur, base);
                rows[static_cast<size_t>(255 * i + v - 1)] = cur;
            }
        });
    for (auto& t : th) t.join();
    for (int r = 0; r < kDigitRows; ++r) {
        to_rows(rows[static_cast<size_t>(r)], &host[static_cast<size_t>(r) * vmt::kPolyWords]);
        c.row_deg[static_cast<size_t>(16 + r)] = vmt::gf2::degree(rows[static_cast<size_t>(r)]);
    }
    CUDA_TRY(cudaMemcpy(c.d_table + 16 * static_cast<size_t>(vmt::kPolyWords), host.data(),
                        host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(c.d_row_deg, c.row_deg.data(), c.row_deg.size() * sizeof(int), cudaMemcpyHostToDevice));
    c.digits_ready = true;
    return VMT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// state object
// ---------------------------------------------------------------------------
// struct vmt_state is defined in vmt_internal.hpp

namespace {

int64_t state_total_bytes(const vmt_state* st) { return st->count * vmt::state_bytes_per_gen(st->variant, st->lanes); }

int run_jump_grid(int variant, const vmt::JumpGrid& gr, long long nitems, const uint32_t* table, cudaStream_t s,
                  int shared = 0)
{
    CUDA_TRY(vmt::launch_jump_grid(variant, gr, nitems, table, s, shared));
    return VMT_OK;
}

int64_t new_block_pos(int64_t B, int64_t p, int64_t total)
{
    if (total <= 0) return p;
    int64_t first = (p < B) ? std::min(B - p, total) : 0;
    int64_t rem = total - first;
    if (rem == 0) return p + first;
    const int64_t nblocks = (rem + B - 1) / B;
    return rem - (nblocks - 1) * B;
}

// advance the host copy of the positions of generators [g0, g0+gens) by `words`
void advance_positions(vmt_state* st, int64_t g0, int64_t gens, int64_t words)
{
    const int64_t B = vmt::block_words(st->variant, st->lanes);
    for (int64_t g = g0; g < g0 + gens; ++g) st->h_pos[static_cast<size_t>(g)] = new_block_pos(B, st->h_pos[static_cast<size_t>(g)], words);
}

void refresh_uniform(vmt_state* st)
{
    st->uniform = true;
    for (size_t g = 1; g < st->h_pos.size() && st->uniform; ++g) st->uniform = st->h_pos[g] == st->h_pos[0];
}

bool range_uniform(const vmt_state* st, int64_t g0, int64_t gens)
{
    if (st->uniform) return true;
    for (int64_t g = g0 + 1; g < g0 + gens; ++g)
        if (st->h_pos[static_cast<size_t>(g)] != st->h_pos[static_cast<size_t>(g0)]) return false;
    return true;
}

bool any_odd(const vmt_state* st, int64_t g0, int64_t gens, int64_t w)
{
    if (st->uniform) return ((st->h_pos[0] + w) & 1) != 0;
    for (int64_t g = g0; g < g0 + gens; ++g)
        if (((st->h_pos[static_cast<size_t>(g)] + w) & 1) != 0) return true;
    return false;
}

int words_per_output(int variant, int dtype)
{
    if (variant == VMT_MT19937_64) return 1;
    return (dtype == VMT_U64 || dtype == VMT_F64) ? 2 : 1;
}

int elem_bytes(int dtype) { return (dtype == VMT_U32 || dtype == VMT_F32) ? 4 : 8; }

int vector_width(int variant, int lanes)
{
    if (variant == VMT_SFMT19937) return 4;
    if (variant == VMT_MT19937_32) return std::min(lanes, 4);
    return std::min(lanes, 2);
}

constexpr int64_t kMaxUnitWords = int64_t(1) << 30;

// grow a pinned host buffer and a device buffer of unit descriptors
int reserve_units(vmt::UnitDesc** h, vmt::UnitDesc** d, int** counter, int64_t* cap, cudaEvent_t* free_ev,
                  int64_t n)
{
    if (!*free_ev) CUDA_TRY(cudaEventCreateWithFlags(free_ev, cudaEventDisableTiming));
    CUDA_TRY(cudaEventSynchronize(*free_ev));   // the previous upload has been read
    if (n > *cap) {
        if (*h) cudaFreeHost(*h);
        if (*d) cudaFree(*d);
        *h = nullptr;
        *d = nullptr;
        const int64_t c = std::max<int64_t>(n, 64);
        CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(h), static_cast<size_t>(c) * sizeof(vmt::UnitDesc), 0));
        CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(d), static_cast<size_t>(c) * sizeof(vmt::UnitDesc)));
        *cap = c;
    }
    if (!*counter) CUDA_TRY(cudaMalloc(reinterpret_cast<void**>(counter), 16 * sizeof(int)));
    return VMT_OK;
}

}  // namespace

int vmt::launch_unit_table(int variant, int lanes, int dtype, const vmt::UnitDesc* d_units, int64_t n, int* counter,
                           void* stream, bool cta_per_unit)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 0) return VMT_OK;
    vmt::GenArgs a{};
    a.gens = n;
    a.kcfg = vmt::tuned_kcfg(variant, lanes);
    a.nseg = 1;
    a.seg[0].dtype = dtype;
    a.seg[0].wbeg = 0;
    a.seg[0].wend = kMaxUnitWords;
    a.units = d_units;
    a.work_counter = counter;
    a.cta_per_unit = cta_per_unit ? 1 : 0;
    CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), s));
    CUDA_TRY(vmt::launch_generate(variant, lanes, a, true, s));
    return VMT_OK;
}

namespace {

int launch_units(int variant, int lanes, int dtype, const vmt::UnitDesc* d_units, int64_t n, int* counter,
                 cudaStream_t s)
{
    return vmt::launch_unit_table(variant, lanes, dtype, d_units, n, counter, s);
}

// Generate `nseg` consecutive segments for generators [g0, g0 + gens) of st,
// whose outputs start at outs[i] (generator g0 writes at outs[i] + 0).  The
// block position is not advanced: all generator ranges of one call start at the
// same position and the caller advances it once.
int generate_range(vmt_state* st, int64_t g0, int64_t gens, int nseg, const int64_t* counts, const int* dtypes,
                   void* const* outs, cudaStream_t s)
{
    if (!st) return fail(VMT_EINVAL, "null state");
    if (nseg < 1 || nseg > VMT_MAXSEG) return fail(VMT_EINVAL, "nseg must be in 1..4");
    const int v = st->variant;
    vmt::GenArgs a{};
    a.states = static_cast<char*>(st->d_states) + g0 * vmt::state_bytes_per_gen(v, st->lanes);
    a.gens = gens;
    a.gen0 = 0;
    a.kcfg = vmt::tuned_kcfg(v, st->lanes);
    a.pos_dev = st->d_pos + g0;
    a.pos = static_cast<int>(st->h_pos[static_cast<size_t>(g0)]);
    a.nseg = nseg;
    const bool ragged = !range_uniform(st, g0, gens);
    int64_t w = 0;
    bool generic = false;
    for (int i = 0; i < nseg; ++i) {
        const int dt = dtypes[i];
        if (dt < VMT_U32 || dt > VMT_F64) return fail(VMT_EINVAL, "bad dtype");
        if (v == VMT_MT19937_64 && dt == VMT_U32) return fail(VMT_EINVAL, "u32 output is not defined for MT19937-64");
        if (counts[i] < 0) return fail(VMT_EINVAL, "negative count");
        if (counts[i] > 0 && !outs[i]) return fail(VMT_EINVAL, "null output pointer");
        const int wpo = words_per_output(v, dt);
        vmt::SegArg& sg = a.seg[i];
        sg.out = static_cast<char*>(outs[i]);
        sg.count = counts[i];
        sg.wbeg = w;
        sg.wend = w + counts[i] * wpo;
        sg.dtype = dt;
        const int eb = elem_bytes(dt);
        sg.fast = ((reinterpret_cast<uintptr_t>(outs[i]) & 15u) == 0 && ((counts[i] * eb) % 16) == 0) ? 1 : 0;
        if (wpo == 2 && counts[i] > 0) {
            // a pair must sit inside one thread's vector: even absolute start and
            // vectors of at least two words
            if (any_odd(st, g0, gens, w) || vector_width(v, st->lanes) < 2) generic = true;
        }
        w += counts[i] * wpo;
    }
    a.total = w;
    if (w == 0 || gens == 0) return VMT_OK;
    if (ragged) {
        // generators at different positions: one unit launch per segment, each
        // generator a unit of that segment's length (positions advance on the
        // device from one segment to the next)
        if (generic) return fail(VMT_EINVAL, "two-word outputs need even stream positions when generators differ");
        int rc = reserve_units(&st->h_units, &st->d_units, &st->d_counter, &st->units_cap, &st->units_free, gens);
        if (rc) return rc;
        const int64_t gen_bytes = vmt::state_bytes_per_gen(v, st->lanes);
        for (int i = 0; i < nseg; ++i) {
            const vmt::SegArg& sg = a.seg[i];
            const int64_t sw = sg.wend - sg.wbeg;
            if (sw == 0) continue;
            if (sw > kMaxUnitWords) return fail(VMT_EINVAL, "segment too long for generators at different positions");
            CUDA_TRY(cudaEventSynchronize(st->units_free));
            for (int64_t g = 0; g < gens; ++g) {
                vmt::UnitDesc& u = st->h_units[g];
                u.state = static_cast<char*>(st->d_states) + (g0 + g) * gen_bytes;
                u.pos = st->d_pos + g0 + g;
                u.total = sw;
                u.out = sg.out + g * sg.count * elem_bytes(sg.dtype);
            }
            CUDA_TRY(cudaMemcpyAsync(st->d_units, st->h_units, static_cast<size_t>(gens) * sizeof(vmt::UnitDesc),
                                     cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaEventRecord(st->units_free, s));
            rc = launch_units(v, st->lanes, sg.dtype, st->d_units, gens, st->d_counter, s);
            if (rc) return rc;
        }
        return VMT_OK;
    }
    // the kernels index words of one call with 32-bit integers: longer calls
    // are cut into pieces of at most 2^30 words (an even number, so that no
    // output pair is split); each piece starts where the previous one ended
    constexpr int64_t kPiece = int64_t(1) << 30;
    if (!generic && w > kPiece) {
        int64_t pos = a.pos;
        const int64_t B = vmt::block_words(v, st->lanes);
        for (int64_t w0 = 0; w0 < w; w0 += kPiece) {
            const int64_t w1 = std::min(w, w0 + kPiece);
            vmt::GenArgs pa = a;
            pa.pos = static_cast<int>(pos);
            pa.total = w1 - w0;
            pos = new_block_pos(B, pos, w1 - w0);
            pa.nseg = 0;
            for (int i = 0; i < nseg; ++i) {
                const vmt::SegArg& sg = a.seg[i];
                const int64_t lo = std::max<int64_t>(sg.wbeg, w0), hi = std::min<int64_t>(sg.wend, w1);
                if (lo >= hi) continue;
                const int wpo = words_per_output(v, sg.dtype);
                vmt::SegArg q = sg;
                // outputs of generator g in this piece start at out + g*count + (lo - wbeg)/wpo;
                // the kernel adds g*count itself
                q.out = sg.out + ((lo - sg.wbeg) / wpo) * elem_bytes(sg.dtype);
                q.wbeg = lo - w0;
                q.wend = hi - w0;
                pa.seg[pa.nseg++] = q;
            }
            CUDA_TRY(vmt::launch_generate(v, st->lanes, pa, ragged, s));
        }
        return VMT_OK;
    }
    if (generic && w > kPiece)
        return fail(VMT_EINVAL, "two-word outputs at an odd word offset are limited to 2^30 words per call");
    if (!generic) {
        CUDA_TRY(vmt::launch_generate(v, st->lanes, a, ragged, s));
    } else {
        // raw native words into scratch, then one conversion per segment
        const int wb = vmt::word_bytes(v);
        void* scratch = nullptr;
        CUDA_TRY(cudaMallocAsync(&scratch, static_cast<size_t>(gens * w * wb), s));
        vmt::GenArgs r = a;
        r.nseg = 1;
        r.seg[0].out = static_cast<char*>(scratch);
        r.seg[0].count = w;
        r.seg[0].wbeg = 0;
        r.seg[0].wend = w;
        r.seg[0].dtype = (v == VMT_MT19937_64) ? VMT_U64 : VMT_U32;
        r.seg[0].fast = 0;
        CUDA_TRY(vmt::launch_generate(v, st->lanes, r, ragged, s));
        for (int i = 0; i < nseg; ++i)
            CUDA_TRY(vmt::launch_convert(scratch, w, v == VMT_MT19937_64, gens, a.seg[i].wbeg, a.seg[i].dtype,
                                         a.seg[i].count, a.seg[i].out, s));
        CUDA_TRY(cudaFreeAsync(scratch, s));
    }
    return VMT_OK;
}

int64_t call_words(const vmt_state* st, int nseg, const int64_t* counts, const int* dtypes)
{
    int64_t w = 0;
    for (int i = 0; i < nseg; ++i) w += counts[i] * words_per_output(st->variant, dtypes[i]);
    return w;
}

int generate_impl(vmt_state* st, int nseg, const int64_t* counts, const int* dtypes, void* const* outs,
                  cudaStream_t s)
{
    if (!st) return fail(VMT_EINVAL, "null state");
    const int rc = generate_range(st, 0, st->count, nseg, counts, dtypes, outs, s);
    if (rc) return rc;
    advance_positions(st, 0, st->count, call_words(st, nseg, counts, dtypes));
    return VMT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char* vmt_last_error(void) { return g_err.c_str(); }

int vmt_set_cache_dir(const char* path)
{
    std::lock_guard<std::mutex> lk(g_cache_lock);
    g_cache_dir = path ? std::string(path) : std::string();
    return VMT_OK;
}

}  // extern "C"

// Creates nsub state objects of one variant (object i: lanes[i] lanes,
// counts[i] generators, whose seeds and offsets follow those of objects
// 0..i-1 in seeds/jumps).  Seeding and the jump offsets run once over all
// generators; the lane fan-out runs per object.  With async_alloc the device
// memory comes from the stream-ordered pool `pool` (the default pool when
// null); free such objects with vmt::free_state_async.
int vmt::init_multi_impl(vmt_state** outs, int variant, int nsub, const int* lanes, const int64_t* counts,
                         const uint64_t* seeds, const uint64_t* jumps, void* cuda_stream, bool async_alloc,
                         cudaMemPool_t pool, int shared_jumps)
{
    if (!outs || !lanes || !counts || nsub < 1) return fail(VMT_EINVAL, "null argument");
    for (int i = 0; i < nsub; ++i) outs[i] = nullptr;
    if (!valid_variant(variant)) return fail(VMT_EINVAL, "bad variant");
    int64_t total = 0;
    for (int i = 0; i < nsub; ++i) {
        if (!valid_lanes(lanes[i])) return fail(VMT_EINVAL, "lanes must be 1, 2, 4, 8 or 16");
        if (counts[i] < 1) return fail(VMT_EINVAL, "count must be >= 1");
        total += counts[i];
    }
    if (!seeds) return fail(VMT_EINVAL, "seeds must be non-null");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = ensure_variant(variant, s);
    if (rc) return rc;
    bool any_jump = false;
    if (jumps)
        for (int64_t g = 0; g < total && !any_jump; ++g) any_jump = jumps[g] != 0;
    if (any_jump && (rc = ensure_digits(variant))) return rc;
    VariantCtx& c = g_ctx[variant];

    std::vector<std::unique_ptr<vmt_state>> made;
    // on any failure below, every object made so far is released
    auto drop = [&](vmt_state* st) { st->async_alloc ? vmt::free_state_async(st, s) : vmt_free(st); };
    const int rc_body = [&]() -> int {
    for (int i = 0; i < nsub; ++i) {
        std::unique_ptr<vmt_state> st(new vmt_state());
        st->variant = variant;
        st->lanes = lanes[i];
        st->count = counts[i];
        CUDA_TRY(cudaGetDevice(&st->device));
        const int64_t bytes = state_total_bytes(st.get());
        const int64_t B = vmt::block_words(variant, lanes[i]);
        bool ok;
        if (async_alloc) {
            ok = vmt::malloc_async(&st->d_states, static_cast<size_t>(bytes), pool, s) == cudaSuccess &&
                 vmt::malloc_async(reinterpret_cast<void**>(&st->d_pos), static_cast<size_t>(counts[i]) * sizeof(int),
                                   pool, s) == cudaSuccess;
            st->async_alloc = true;
        } else {
            ok = cudaMalloc(&st->d_states, static_cast<size_t>(bytes)) == cudaSuccess &&
                 cudaMalloc(reinterpret_cast<void**>(&st->d_pos), static_cast<size_t>(counts[i]) * sizeof(int)) ==
                     cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            drop(st.release());
            return fail(VMT_ENOMEM, "allocation of " + std::to_string(bytes) + " state bytes failed");
        }
        st->h_pos.assign(static_cast<size_t>(counts[i]), B);   // exhausted: the first output twists
        st->uniform = true;
        CUDA_TRY(vmt::launch_fill_int(st->d_pos, counts[i], static_cast<int>(B), s));
        made.push_back(std::move(st));
    }
    const int n_units = vmt::units_per_lane(variant);
    const int unit_bytes = vmt::word_bytes(variant) * vmt::words_per_unit(variant);
    // scratch: seeds, offsets and the unjumped base states, unit-major [u][g]
    unsigned long long* d_seeds = nullptr;
    unsigned long long* d_jumps = nullptr;
    char* d_base = nullptr;
    CUDA_TRY(vmt::malloc_async(reinterpret_cast<void**>(&d_seeds), static_cast<size_t>(total) * 8, pool, s));
    CUDA_TRY(vmt::malloc_async(reinterpret_cast<void**>(&d_base), static_cast<size_t>(total * n_units * unit_bytes),
                               pool, s));
    CUDA_TRY(cudaMemcpyAsync(d_seeds, seeds, static_cast<size_t>(total) * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(vmt::launch_seed(variant, total, d_seeds, d_base, s));
    vmt::JumpGrid gr{};
    gr.count = total;
    gr.base = d_base;
    gr.unit_bytes = unit_bytes;
    gr.row_deg = c.d_row_deg;
    if (any_jump) {
        // base <- x^d(F) base, one base-256 digit per launch (jumps commute)
        CUDA_TRY(vmt::malloc_async(reinterpret_cast<void**>(&d_jumps), static_cast<size_t>(total) * 8, pool, s));
        CUDA_TRY(cudaMemcpyAsync(d_jumps, jumps, static_cast<size_t>(total) * 8, cudaMemcpyHostToDevice, s));
        gr.mode = vmt::JumpGrid::kDigit;
        gr.jumps = d_jumps;
        for (int i = 0; i < 8; ++i) {
            bool used = false;
            for (int64_t g = 0; g < total && !used; ++g) used = ((jumps[g] >> (8 * i)) & 255u) != 0;
            if (!used) continue;
            gr.digit = i;
            if ((rc = run_jump_grid(variant, gr, total, c.d_table, s, shared_jumps))) return rc;
        }
    }
    // lane fan-out per object: lane t = x^(t J)(F) base, written into X-hat's
    // column t (the base keeps its unit stride `total`)
    gr.mode = vmt::JumpGrid::kFanOut;
    int64_t g0 = 0;
    for (int i = 0; i < nsub; ++i) {
        gr.base = d_base + g0 * unit_bytes;
        gr.lanes = lanes[i];
        gr.states = static_cast<char*>(made[static_cast<size_t>(i)]->d_states);
        gr.gen_bytes = vmt::state_bytes_per_gen(variant, lanes[i]);
        if ((rc = run_jump_grid(variant, gr, counts[i] * lanes[i], c.d_table, s, shared_jumps))) return rc;
        g0 += counts[i];
    }
    CUDA_TRY(cudaFreeAsync(d_seeds, s));
    CUDA_TRY(cudaFreeAsync(d_base, s));
    if (d_jumps) CUDA_TRY(cudaFreeAsync(d_jumps, s));
    return VMT_OK;
    }();
    if (rc_body != VMT_OK) {
        for (auto& m : made) drop(m.release());
        return rc_body;
    }
    for (int i = 0; i < nsub; ++i) outs[i] = made[static_cast<size_t>(i)].release();
    return VMT_OK;
}

int vmt::init_batch_impl(vmt_state** out, int variant, int lanes, int64_t count, const uint64_t* seeds,
                         const uint64_t* jumps, void* cuda_stream, bool async_alloc, cudaMemPool_t pool)
{
    if (!out) return fail(VMT_EINVAL, "null output handle");
    return vmt::init_multi_impl(out, variant, 1, &lanes, &count, seeds, jumps, cuda_stream, async_alloc, pool);
}

int vmt::alloc_states_async(vmt_state** out, int variant, int lanes, int64_t count, void* cuda_stream,
                            cudaMemPool_t pool)
{
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    std::unique_ptr<vmt_state> st(new vmt_state());
    st->variant = variant;
    st->lanes = lanes;
    st->count = count;
    st->async_alloc = true;
    CUDA_TRY(cudaGetDevice(&st->device));
    const int64_t B = vmt::block_words(variant, lanes);
    if (vmt::malloc_async(&st->d_states, static_cast<size_t>(state_total_bytes(st.get())), pool, s) != cudaSuccess ||
        vmt::malloc_async(reinterpret_cast<void**>(&st->d_pos), static_cast<size_t>(count) * sizeof(int), pool, s) !=
            cudaSuccess) {
        cudaGetLastError();
        if (st->d_states) cudaFreeAsync(st->d_states, s);
        return fail(VMT_ENOMEM, "chunk state allocation failed");
    }
    st->h_pos.assign(static_cast<size_t>(count), B);
    CUDA_TRY(vmt::launch_fill_int(st->d_pos, count, static_cast<int>(B), s));
    *out = st.release();
    return VMT_OK;
}

int vmt::launch_chunk_jumps(const vmt_state* requests, vmt_state* chunks, const int2* d_map, void* cuda_stream,
                            int shared_jumps)
{
    const int variant = requests->variant;
    int rc = ensure_chunks(variant);
    if (rc) return rc;
    VariantCtx& c = g_ctx[variant];
    vmt::JumpGrid gr{};
    gr.mode = vmt::JumpGrid::kChunk;
    gr.count = chunks->count;
    gr.lanes = requests->lanes;
    gr.base = static_cast<char*>(requests->d_states);
    gr.unit_bytes = vmt::word_bytes(variant) * vmt::words_per_unit(variant);
    gr.states = static_cast<char*>(chunks->d_states);
    gr.gen_bytes = vmt::state_bytes_per_gen(variant, requests->lanes);
    gr.row_deg = c.d_row_deg;
    gr.chunk_map = d_map;
    gr.chunk_row0 = kChunkRow0;
    return run_jump_grid(variant, gr, chunks->count * requests->lanes, c.d_table, static_cast<cudaStream_t>(cuda_stream),
                         shared_jumps);
}

void vmt::free_state_async(vmt_state* st, void* cuda_stream)
{
    if (!st) return;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (st->d_states) cudaFreeAsync(st->d_states, s);
    if (st->d_pos) cudaFreeAsync(st->d_pos, s);
    st->d_states = nullptr;
    st->d_pos = nullptr;
    vmt_free(st);
}

extern "C" {

int vmt_init_batch(vmt_state** out, int variant, int lanes, int64_t count, const uint64_t* seeds,
                   const uint64_t* jumps, void* cuda_stream)
{
    return vmt::init_batch_impl(out, variant, lanes, count, seeds, jumps, cuda_stream, false);
}

int vmt_init(vmt_state** st, int variant, int lanes, uint64_t seed, uint64_t jump, void* cuda_stream)
{
    return vmt_init_batch(st, variant, lanes, 1, &seed, &jump, cuda_stream);
}

int vmt_jump(vmt_state* st, const uint64_t* poly, int64_t nbits, void* cuda_stream)
{
    if (!st || !poly) return fail(VMT_EINVAL, "null argument");
    if (nbits < 0 || nbits > 32 * vmt::kPolyWords - 64) return fail(VMT_EINVAL, "nbits out of range");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // one device row holding the polynomial, followed by its degree
    std::vector<uint32_t> row(static_cast<size_t>(vmt::kPolyWords) + 1, 0);
    const int64_t nw = (nbits + 63) / 64;
    Poly p(poly, poly + nw);
    if (nbits % 64 && nw) p[static_cast<size_t>(nw - 1)] &= (1ull << (nbits % 64)) - 1;
    to_rows(p, row.data());
    const int deg = vmt::gf2::degree(p);
    std::memcpy(&row[static_cast<size_t>(vmt::kPolyWords)], &deg, sizeof(int));
    uint32_t* d_row = nullptr;
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_row), row.size() * 4, s));
    CUDA_TRY(cudaMemcpyAsync(d_row, row.data(), row.size() * 4, cudaMemcpyHostToDevice, s));
    // every lane of every generator in place: the fan-out formula with the
    // base being X-hat itself (unit stride = lanes) and row 0 for every lane
    std::vector<vmt::JumpItem> items;
    const int unit_bytes = vmt::word_bytes(st->variant) * vmt::words_per_unit(st->variant);
    const int64_t gen_bytes = vmt::state_bytes_per_gen(st->variant, st->lanes);
    items.reserve(static_cast<size_t>(st->count * st->lanes));
    for (int64_t g = 0; g < st->count; ++g)
        for (int t = 0; t < st->lanes; ++t) {
            vmt::JumpItem it{};
            it.src = static_cast<char*>(st->d_states) + g * gen_bytes + t * unit_bytes;
            it.dst = const_cast<void*>(it.src);
            it.src_stride = st->lanes;
            it.dst_stride = st->lanes;
            it.poly = 0;
            it.deg = deg;
            items.push_back(it);
        }
    vmt::JumpItem* d_items = nullptr;
    const size_t ib = items.size() * sizeof(vmt::JumpItem);
    CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_items), ib, s));
    CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), ib, cudaMemcpyHostToDevice, s));
    CUDA_TRY(vmt::launch_jump(st->variant, d_items, static_cast<long long>(items.size()), d_row, s));
    CUDA_TRY(cudaFreeAsync(d_items, s));
    CUDA_TRY(cudaFreeAsync(d_row, s));
    // the host vectors were staged by the copies above (pageable memory)
    return VMT_OK;
}

// ---------------------------------------------------------------------------
// exact single-stream mode
// ---------------------------------------------------------------------------
// One base generator's stream (M = 1) cut into P chunks of equal length; chunk
// j's state is the base state advanced by j chunk lengths.  The chunk states
// come from a doubling tree of jumps (Sec. 3.1): at level k, chunk j in
// [2^k, 2^(k+1)) is chunk j - 2^k jumped by x^(2^k * steps), so only the
// polynomials x^(2^k * steps) mod mu, k < log2 P, are needed (one power, then
// squarings; cached per variant and chunk length).
namespace {
struct StreamPolys {
    uint64_t steps = 0;
    std::vector<Poly> rows;
};
std::mutex g_stream_mu;
StreamPolys g_stream_polys[3];

void stream_polys(int variant, uint64_t steps, int levels, std::vector<Poly>& out)
{
    VariantCtx& c = g_ctx[variant];
    std::lock_guard<std::mutex> lk(g_stream_mu);
    StreamPolys& sp = g_stream_polys[variant];
    if (sp.steps != steps) {
        sp.steps = steps;
        sp.rows.clear();
    }
    if (sp.rows.empty()) sp.rows.push_back(c.mod->x_pow(steps));
    while (static_cast<int>(sp.rows.size()) < levels) sp.rows.push_back(c.mod->sqr(sp.rows.back()));
    out.assign(sp.rows.begin(), sp.rows.begin() + levels);
}
}  // namespace

int vmt_stream_generate(int variant, uint64_t seed, uint64_t jump, int64_t n, int dtype, void* out_dev,
                        void* cuda_stream)
{
    if (!valid_variant(variant)) return fail(VMT_EINVAL, "bad variant");
    const bool type_ok = variant == VMT_MT19937_64 ? (dtype == VMT_U64 || dtype == VMT_F64 || dtype == VMT_F32)
                                                   : (dtype == VMT_U32 || dtype == VMT_F32);
    if (!type_ok) return fail(VMT_EINVAL, "output type must take one word of the generator");
    if (n < 0 || n > (int64_t(1) << 39)) return fail(VMT_EINVAL, "n must be in 0 .. 2^39");
    if (n > 0 && !out_dev) return fail(VMT_EINVAL, "null output");
    if (n == 0) return VMT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t B = vmt::block_words(variant, 1);
    const int64_t blocks = (n + B - 1) / B;
    // up to 2048 chunks (one warp or a few threads each), at least 64 blocks long
    const int64_t chunk_blocks = std::max<int64_t>(64, (blocks + 2047) / 2048);
    const int64_t P = (blocks + chunk_blocks - 1) / chunk_blocks;   // <= 2048
    const int64_t chunk_words = chunk_blocks * B;
    int levels = 0;
    while ((int64_t(1) << levels) < P) ++levels;
    const int64_t gen_bytes = vmt::state_bytes_per_gen(variant, 1);

    // chunk 0: the base generator advanced by `jump` (seeding as vmt_init)
    vmt_state* st0 = nullptr;
    int rc = vmt::init_batch_impl(&st0, variant, 1, 1, &seed, &jump, s, true);
    if (rc) return rc;
    vmt_state* cs = nullptr;
    rc = vmt::alloc_states_async(&cs, variant, 1, P, s);
    if (rc) {
        vmt::free_state_async(st0, s);
        return rc;
    }
    uint32_t* d_rows = nullptr;
    vmt::JumpItem* d_items = nullptr;
    vmt::UnitDesc* d_units = nullptr;
    int* d_counter = nullptr;
    rc = [&]() -> int {
        CUDA_TRY(cudaMemcpyAsync(cs->d_states, st0->d_states, static_cast<size_t>(gen_bytes), cudaMemcpyDeviceToDevice,
                                 s));
        if (P > 1) {
            std::vector<Poly> polys;
            stream_polys(variant, static_cast<uint64_t>(chunk_blocks) * vmt::units_per_lane(variant), levels, polys);
            std::vector<uint32_t> rows(static_cast<size_t>(levels) * vmt::kPolyWords, 0);
            std::vector<int> deg(static_cast<size_t>(levels));
            for (int k = 0; k < levels; ++k) {
                to_rows(polys[static_cast<size_t>(k)], &rows[static_cast<size_t>(k) * vmt::kPolyWords]);
                deg[static_cast<size_t>(k)] = vmt::gf2::degree(polys[static_cast<size_t>(k)]);
            }
            CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_rows), rows.size() * 4, s));
            CUDA_TRY(cudaMemcpyAsync(d_rows, rows.data(), rows.size() * 4, cudaMemcpyHostToDevice, s));
            // level k: chunks [2^k, min(2^(k+1), P)) from chunks 2^k earlier
            std::vector<vmt::JumpItem> items;
            std::vector<std::pair<int64_t, int64_t>> level_range;
            char* base = static_cast<char*>(cs->d_states);
            for (int k = 0; k < levels; ++k) {
                const int64_t lo = int64_t(1) << k, hi = std::min<int64_t>(int64_t(2) << k, P);
                level_range.push_back({static_cast<int64_t>(items.size()), hi - lo});
                for (int64_t j = lo; j < hi; ++j) {
                    vmt::JumpItem it{};
                    it.src = base + (j - lo) * gen_bytes;
                    it.dst = base + j * gen_bytes;
                    it.src_stride = 1;
                    it.dst_stride = 1;
                    it.poly = k;
                    it.deg = deg[static_cast<size_t>(k)];
                    items.push_back(it);
                }
            }
            CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_items), items.size() * sizeof(vmt::JumpItem), s));
            CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(vmt::JumpItem),
                                     cudaMemcpyHostToDevice, s));
            for (const auto& lr : level_range)
                CUDA_TRY(vmt::launch_jump(variant, d_items + lr.first, static_cast<long long>(lr.second), d_rows, s));
        }
        // one unit per chunk; the last one takes the rest
        std::vector<vmt::UnitDesc> units(static_cast<size_t>(P));
        const int64_t eb = elem_bytes(dtype);
        for (int64_t j = 0; j < P; ++j) {
            vmt::UnitDesc& u = units[static_cast<size_t>(j)];
            u.state = static_cast<char*>(cs->d_states) + j * gen_bytes;
            u.pos = cs->d_pos + j;
            u.total = std::min<int64_t>(chunk_words, n - j * chunk_words);
            u.out = static_cast<char*>(out_dev) + j * chunk_words * eb;
        }
        CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_units), units.size() * sizeof(vmt::UnitDesc), s));
        CUDA_TRY(cudaMemcpyAsync(d_units, units.data(), units.size() * sizeof(vmt::UnitDesc), cudaMemcpyHostToDevice,
                                 s));
        CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d_counter), sizeof(int), s));
        return vmt::launch_unit_table(variant, 1, dtype, d_units, P, d_counter, s);
    }();
    if (d_rows) cudaFreeAsync(d_rows, s);
    if (d_items) cudaFreeAsync(d_items, s);
    if (d_units) cudaFreeAsync(d_units, s);
    if (d_counter) cudaFreeAsync(d_counter, s);
    vmt::free_state_async(st0, s);
    vmt::free_state_async(cs, s);
    return rc;
}

int vmt_tune_jump_set(int variant, int64_t split_below)
{
    if (split_below < 0) return fail(VMT_EINVAL, "split_below must be >= 0");
    if (variant != -1 && !valid_variant(variant)) return fail(VMT_EINVAL, "bad variant");
    for (int v = 0; v < 3; ++v)
        if (variant == -1 || variant == v) vmt::set_jump_split_below(v, split_below);
    return VMT_OK;
}

int64_t vmt_tune_jump_get(int variant)
{
    if (!valid_variant(variant)) return fail(VMT_EINVAL, "bad variant");
    return vmt::get_jump_split_below(variant);
}

int vmt_tune_jump_compact(int variant, int on)
{
    if (variant < -1 || variant > 2 || on < -1 || on > 1) return fail(VMT_EINVAL, "bad variant or setting");
    const int old = vmt::get_jump_compact(variant < 0 ? 0 : variant);
    if (on >= 0)
        for (int v = 0; v < 3; ++v)
            if (variant < 0 || v == variant) vmt::set_jump_compact(v, on);
    return old;
}

int vmt_prepare(int variant, void* cuda_stream)
{
    if (!valid_variant(variant)) return fail(VMT_EINVAL, "bad variant");
    int rc = ensure_variant(variant, static_cast<cudaStream_t>(cuda_stream));
    if (!rc) rc = ensure_digits(variant);
    if (!rc) rc = ensure_chunks(variant);
    return rc;
}

int vmt_jump_poly(int variant, uint64_t d, int log2_extra, uint64_t* poly_out, int64_t cap_words)
{
    if (!valid_variant(variant) || !poly_out || log2_extra < 0) return fail(VMT_EINVAL, "bad argument");
    int rc = ensure_variant(variant, nullptr);
    if (rc) return rc;
    VariantCtx& c = g_ctx[variant];
    // x^(d 2^e) = (x^d)^(2^e): e squarings of x^d, x^d being the product of the
    // stored chain entries x^(2^q) at the set bits q of d, multiplied as a
    // balanced tree whose products of one level run on separate threads
    std::vector<Poly> f;
    for (int q = 0; q < 64; ++q)
        if ((d >> q) & 1ull) f.push_back(c.chain_lo[static_cast<size_t>(q)]);
    if (f.empty()) f.push_back(c.mod->reduce(Poly(1, 1)));
    while (f.size() > 1) {
        std::vector<Poly> g((f.size() + 1) / 2);
        std::vector<std::thread> th;
        for (size_t i = 0; i + 1 < f.size(); i += 2)
            th.emplace_back([&, i]() { g[i / 2] = c.mod->mul(f[i], f[i + 1]); });
        if (f.size() % 2) g.back() = f.back();
        for (auto& t : th) t.join();
        f.swap(g);
    }
    Poly r = f[0];
    for (int i = 0; i < log2_extra; ++i) r = c.mod->sqr(r);
    const int64_t nw = static_cast<int64_t>(r.size());
    if (cap_words < nw) return fail(VMT_EINVAL, "poly_out too small");
    std::memset(poly_out, 0, static_cast<size_t>(cap_words) * 8);
    std::memcpy(poly_out, r.data(), static_cast<size_t>(nw) * 8);
    return static_cast<int>(nw);
}

int vmt_generate_multi(vmt_state* st, int nseg, const int64_t* counts, const int* dtypes, void* const* outs,
                       void* cuda_stream)
{
    if (!counts || !dtypes || !outs) return fail(VMT_EINVAL, "null segment arrays");
    return generate_impl(st, nseg, counts, dtypes, outs, static_cast<cudaStream_t>(cuda_stream));
}

int vmt_generate(vmt_state* st, int64_t n, int dtype, void* out_dev, void* cuda_stream)
{
    void* outs[1] = {out_dev};
    return generate_impl(st, 1, &n, &dtype, outs, static_cast<cudaStream_t>(cuda_stream));
}

int vmt_generate_host(vmt_state* st, int64_t n, int dtype, void* out_host, void* cuda_stream)
{
    if (!st || (!out_host && n > 0)) return fail(VMT_EINVAL, "null argument");
    if (n < 0) return fail(VMT_EINVAL, "negative count");
    if (dtype < VMT_U32 || dtype > VMT_F64) return fail(VMT_EINVAL, "bad dtype");
    if (n == 0) return VMT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // Pinned host memory is mapped into the device's address space: the
    // generation kernels store into it directly over the CPU-GPU link, with
    // no staging buffer and no separate copy (on GB300 as fast as the copy
    // engines, which share the same host-memory bandwidth).
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, out_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer != nullptr) {
        int rc = vmt_generate(st, n, dtype, pa.devicePointer, cuda_stream);
        if (rc == VMT_OK) CUDA_TRY(cudaStreamSynchronize(s));
        return rc;
    }
    cudaGetLastError();
    const int64_t eb = elem_bytes(dtype);
    const int64_t row = n * eb;   // one generator's output bytes
    const int64_t kStage = int64_t(256) << 20;
    if (row > kStage) {
        // very long rows: generate the whole call on the device in one pass and
        // copy it back in one piece
        void* buf = nullptr;
        CUDA_TRY(cudaMallocAsync(&buf, static_cast<size_t>(row * st->count), s));
        int rc = vmt_generate(st, n, dtype, buf, s);
        if (rc == VMT_OK) {
            cudaError_t e = cudaMemcpyAsync(out_host, buf, static_cast<size_t>(row * st->count), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) rc = fail(VMT_ECUDA, cudaGetErrorString(e));
        }
        cudaFreeAsync(buf, s);
        return rc;
    }
    // generator ranges: every range produces whole rows, so each device-to-host
    // copy is one contiguous block; two staging buffers alternate so that the
    // copy of one range overlaps the generation of the next
    const int64_t per = std::max<int64_t>(1, std::min<int64_t>(st->count, kStage / row));
    void* stage[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    cudaEvent_t done_gen[2], done_copy[2];
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        CUDA_TRY(cudaMallocAsync(&stage[i], static_cast<size_t>(per * row), s));
        CUDA_TRY(cudaEventCreateWithFlags(&done_gen[i], cudaEventDisableTiming));
        CUDA_TRY(cudaEventCreateWithFlags(&done_copy[i], cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(done_copy[i], cs));
    }
    int rc = VMT_OK;
    int k = 0;
    for (int64_t g0 = 0; g0 < st->count && rc == VMT_OK; g0 += per, ++k) {
        const int b = k & 1;
        const int64_t gens = std::min(per, st->count - g0);
        CUDA_TRY(cudaStreamWaitEvent(s, done_copy[b], 0));
        void* outs[1] = {stage[b]};
        rc = generate_range(st, g0, gens, 1, &n, &dtype, outs, s);
        if (rc) break;
        CUDA_TRY(cudaEventRecord(done_gen[b], s));
        CUDA_TRY(cudaStreamWaitEvent(cs, done_gen[b], 0));
        CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(out_host) + g0 * row, stage[b], static_cast<size_t>(gens * row),
                                 cudaMemcpyDeviceToHost, cs));
        CUDA_TRY(cudaEventRecord(done_copy[b], cs));
    }
    CUDA_TRY(cudaStreamSynchronize(cs));
    for (int i = 0; i < 2; ++i) {
        cudaFreeAsync(stage[i], s);
        cudaEventDestroy(done_gen[i]);
        cudaEventDestroy(done_copy[i]);
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    cudaStreamDestroy(cs);
    if (rc == VMT_OK) advance_positions(st, 0, st->count, n * words_per_output(st->variant, dtype));
    return rc;
}

// ---------------------------------------------------------------------------
// ragged and batched launches (one persistent launch over many generators of
// different lengths; see include/vmt.h)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// checks shared by the ragged and batched forms for generator g of st
int check_unit(const vmt_state* st, int64_t g, int64_t n, int dtype, const void* out)
{
    if (dtype < VMT_U32 || dtype > VMT_F64) return fail(VMT_EINVAL, "bad dtype");
    if (st->variant == VMT_MT19937_64 && dtype == VMT_U32)
        return fail(VMT_EINVAL, "u32 output is not defined for MT19937-64");
    if (n < 0) return fail(VMT_EINVAL, "negative count");
    if (n > 0 && !out) return fail(VMT_EINVAL, "null output pointer");
    const int wpo = words_per_output(st->variant, dtype);
    if (n * wpo > kMaxUnitWords) return fail(VMT_EINVAL, "ragged/batched calls are limited to 2^30 words per generator");
    if (wpo == 2 && n > 0 && ((st->h_pos[static_cast<size_t>(g)] & 1) != 0 || vector_width(st->variant, st->lanes) < 2))
        return fail(VMT_EINVAL,
                    "two-word outputs in ragged/batched calls need an even stream position and at least 2 lanes");
    return VMT_OK;
}

}  // namespace

struct vmt_batch {
    struct Item {
        vmt_state* st;
        int64_t n;
        int dtype;
        char* out;
    };
    std::vector<Item> items;
    // groups of units sharing (variant, lanes, dtype), contiguous in the unit array
    struct Group {
        int variant, lanes, dtype;
        int64_t first, count;
    };
    std::vector<Group> groups;
    vmt::UnitDesc* h_units = nullptr;
    vmt::UnitDesc* d_units = nullptr;
    int* d_counter = nullptr;
    int64_t cap = 0;
    cudaEvent_t free_ev = nullptr;
    bool built = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;
};

namespace {

int batch_build(vmt_batch* b)
{
    // units grouped by kernel, longest first inside a group
    std::vector<std::pair<std::tuple<int, int, int>, vmt::UnitDesc>> all;
    for (const auto& it : b->items) {
        vmt_state* st = it.st;
        const int64_t gen_bytes = vmt::state_bytes_per_gen(st->variant, st->lanes);
        const int64_t words = it.n * words_per_output(st->variant, it.dtype);
        const int eb = elem_bytes(it.dtype);
        if (words == 0) continue;
        for (int64_t g = 0; g < st->count; ++g) {
            vmt::UnitDesc u{};
            u.state = static_cast<char*>(st->d_states) + g * gen_bytes;
            u.pos = st->d_pos + g;
            u.total = words;
            u.out = it.out + g * it.n * eb;
            all.push_back({std::make_tuple(st->variant, st->lanes, it.dtype), u});
        }
    }
    std::stable_sort(all.begin(), all.end(), [](const auto& x, const auto& y) {
        if (x.first != y.first) return x.first < y.first;
        return x.second.total > y.second.total;
    });
    int rc = reserve_units(&b->h_units, &b->d_units, &b->d_counter, &b->cap, &b->free_ev,
                           static_cast<int64_t>(all.size()));
    if (rc) return rc;
    b->groups.clear();
    for (size_t i = 0; i < all.size(); ++i) {
        b->h_units[i] = all[i].second;
        if (b->groups.empty() || std::make_tuple(b->groups.back().variant, b->groups.back().lanes,
                                                 b->groups.back().dtype) != all[i].first) {
            if (b->groups.size() == 16) return fail(VMT_EINVAL, "a batch may mix at most 16 kernel groups");
            b->groups.push_back({std::get<0>(all[i].first), std::get<1>(all[i].first), std::get<2>(all[i].first),
                                 static_cast<int64_t>(i), 0});
        }
        b->groups.back().count++;
    }
    b->built = true;
    return VMT_OK;
}

int batch_enqueue(vmt_batch* b, cudaStream_t s)
{
    const int64_t n = b->groups.empty() ? 0 : b->groups.back().first + b->groups.back().count;
    if (n == 0) return VMT_OK;
    CUDA_TRY(cudaMemcpyAsync(b->d_units, b->h_units, static_cast<size_t>(n) * sizeof(vmt::UnitDesc),
                             cudaMemcpyHostToDevice, s));
    for (size_t k = 0; k < b->groups.size(); ++k) {
        const auto& gr = b->groups[k];
        const int rc = launch_units(gr.variant, gr.lanes, gr.dtype, b->d_units + gr.first, gr.count,
                                    b->d_counter + k, s);
        if (rc) return rc;
    }
    return VMT_OK;
}

void batch_advance(vmt_batch* b)
{
    for (const auto& it : b->items) {
        advance_positions(it.st, 0, it.st->count, it.n * words_per_output(it.st->variant, it.dtype));
        refresh_uniform(it.st);
    }
}

int batch_check(vmt_batch* b)
{
    for (const auto& it : b->items)
        for (int64_t g = 0; g < it.st->count; ++g) {
            const int rc = check_unit(it.st, g, it.n, it.dtype, it.out);
            if (rc) return rc;
        }
    return VMT_OK;
}

void batch_drop_graph(vmt_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

}  // namespace

extern "C" {

int vmt_generate_ragged(vmt_state* st, const int64_t* n, int dtype, void* const* outs, void* cuda_stream)
{
    if (!st || !n || !outs) return fail(VMT_EINVAL, "null argument");
    for (int64_t g = 0; g < st->count; ++g) {
        const int rc = check_unit(st, g, n[g], dtype, outs[g]);
        if (rc) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int rc = reserve_units(&st->h_units, &st->d_units, &st->d_counter, &st->units_cap, &st->units_free, st->count);
    if (rc) return rc;
    const int wpo = words_per_output(st->variant, dtype);
    const int64_t gen_bytes = vmt::state_bytes_per_gen(st->variant, st->lanes);
    int64_t k = 0;
    for (int64_t g = 0; g < st->count; ++g) {
        if (n[g] == 0) continue;
        vmt::UnitDesc& u = st->h_units[k++];
        u.state = static_cast<char*>(st->d_states) + g * gen_bytes;
        u.pos = st->d_pos + g;
        u.total = n[g] * wpo;
        u.out = static_cast<char*>(outs[g]);
    }
    std::stable_sort(st->h_units, st->h_units + k,
                     [](const vmt::UnitDesc& x, const vmt::UnitDesc& y) { return x.total > y.total; });
    CUDA_TRY(cudaMemcpyAsync(st->d_units, st->h_units, static_cast<size_t>(k) * sizeof(vmt::UnitDesc),
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(st->units_free, s));
    rc = launch_units(st->variant, st->lanes, dtype, st->d_units, k, st->d_counter, s);
    if (rc) return rc;
    for (int64_t g = 0; g < st->count; ++g) advance_positions(st, g, 1, n[g] * wpo);
    refresh_uniform(st);
    return VMT_OK;
}

int vmt_batch_create(vmt_batch** b)
{
    if (!b) return fail(VMT_EINVAL, "null handle");
    *b = new vmt_batch();
    return VMT_OK;
}

int vmt_batch_add(vmt_batch* b, vmt_state* st, int64_t n, int dtype, void* out_dev)
{
    if (!b || !st) return fail(VMT_EINVAL, "null argument");
    for (const auto& it : b->items)
        if (it.st == st) return fail(VMT_EINVAL, "a state may appear once per batch");
    for (int64_t g = 0; g < st->count; ++g) {
        const int rc = check_unit(st, g, n, dtype, out_dev);
        if (rc) return rc;
    }
    b->items.push_back({st, n, dtype, static_cast<char*>(out_dev)});
    b->built = false;
    batch_drop_graph(b);
    return VMT_OK;
}

int vmt_batch_run(vmt_batch* b, void* cuda_stream)
{
    if (!b) return fail(VMT_EINVAL, "null batch");
    int rc = batch_check(b);
    if (rc) return rc;
    if (!b->built && (rc = batch_build(b))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if ((rc = batch_enqueue(b, s))) return rc;
    CUDA_TRY(cudaEventRecord(b->free_ev, s));
    batch_advance(b);
    return VMT_OK;
}

int vmt_batch_run_graph(vmt_batch* b, void* cuda_stream)
{
    if (!b) return fail(VMT_EINVAL, "null batch");
    int rc = batch_check(b);
    if (rc) return rc;
    if (!b->built && (rc = batch_build(b))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!b->exec) {
        if (!b->capture_stream) CUDA_TRY(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
        rc = batch_enqueue(b, b->capture_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(VMT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        b->graph = g;
        CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
    CUDA_TRY(cudaGraphLaunch(b->exec, s));
    CUDA_TRY(cudaEventRecord(b->free_ev, s));
    batch_advance(b);
    return VMT_OK;
}

int vmt_batch_clear(vmt_batch* b)
{
    if (!b) return fail(VMT_EINVAL, "null batch");
    b->items.clear();
    b->groups.clear();
    b->built = false;
    batch_drop_graph(b);
    return VMT_OK;
}

void vmt_batch_destroy(vmt_batch* b)
{
    if (!b) return;
    if (b->free_ev) cudaEventSynchronize(b->free_ev), cudaEventDestroy(b->free_ev);
    batch_drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->h_units) cudaFreeHost(b->h_units);
    if (b->d_units) cudaFree(b->d_units);
    if (b->d_counter) cudaFree(b->d_counter);
    delete b;
}

struct ExportHeader {
    char magic[8];
    int32_t version, variant, lanes, pad;
    int64_t count, reserved, state_bytes;
};

int64_t vmt_state_bytes(const vmt_state* st)
{
    if (!st) return fail(VMT_EINVAL, "null state");
    return static_cast<int64_t>(sizeof(ExportHeader)) + state_total_bytes(st) + st->count * 8;
}

int vmt_state_export(const vmt_state* st, void* host_buf, size_t cap, void* cuda_stream)
{
    if (!st || !host_buf) return fail(VMT_EINVAL, "null argument");
    const int64_t need = vmt_state_bytes(st);
    if (static_cast<int64_t>(cap) < need) return fail(VMT_EINVAL, "buffer too small");
    ExportHeader h{};
    std::memcpy(h.magic, "VMTSTAT2", 8);
    h.version = 2;
    h.variant = st->variant;
    h.lanes = st->lanes;
    h.count = st->count;
    h.state_bytes = state_total_bytes(st);
    std::memcpy(host_buf, &h, sizeof(h));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(host_buf) + sizeof(h), st->d_states, static_cast<size_t>(h.state_bytes),
                             cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    // per-generator stream positions follow the states
    std::memcpy(static_cast<char*>(host_buf) + sizeof(h) + h.state_bytes, st->h_pos.data(),
                static_cast<size_t>(st->count) * 8);
    return VMT_OK;
}

int vmt_state_import(vmt_state* st, const void* host_buf, size_t len, void* cuda_stream)
{
    if (!st || !host_buf) return fail(VMT_EINVAL, "null argument");
    if (len < sizeof(ExportHeader)) return fail(VMT_ESTATE, "buffer shorter than the header");
    ExportHeader h{};
    std::memcpy(&h, host_buf, sizeof(h));
    if (std::memcmp(h.magic, "VMTSTAT2", 8) != 0 || h.version != 2) return fail(VMT_ESTATE, "not a vmt state export");
    if (h.variant != st->variant || h.lanes != st->lanes || h.count != st->count ||
        h.state_bytes != state_total_bytes(st))
        return fail(VMT_ESTATE, "export does not match this state object");
    if (static_cast<int64_t>(len) < static_cast<int64_t>(sizeof(h)) + h.state_bytes + h.count * 8)
        return fail(VMT_ESTATE, "truncated export");
    const int64_t B = vmt::block_words(st->variant, st->lanes);
    std::vector<int64_t> pos(static_cast<size_t>(h.count));
    std::memcpy(pos.data(), static_cast<const char*>(host_buf) + sizeof(h) + h.state_bytes, pos.size() * 8);
    std::vector<int> pos32(pos.size());
    for (size_t g = 0; g < pos.size(); ++g) {
        if (pos[g] < 0 || pos[g] > B) return fail(VMT_ESTATE, "block position out of range");
        pos32[g] = static_cast<int>(pos[g]);
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CUDA_TRY(cudaMemcpyAsync(st->d_states, static_cast<const char*>(host_buf) + sizeof(h),
                             static_cast<size_t>(h.state_bytes), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(st->d_pos, pos32.data(), pos32.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    st->h_pos = pos;
    refresh_uniform(st);
    return VMT_OK;
}

int vmt_state_info(const vmt_state* st, int* variant, int* lanes, int64_t* count, int64_t* block_pos)
{
    if (!st) return fail(VMT_EINVAL, "null state");
    if (variant) *variant = st->variant;
    if (lanes) *lanes = st->lanes;
    if (count) *count = st->count;
    if (block_pos) *block_pos = st->h_pos.empty() ? 0 : st->h_pos[0];
    return VMT_OK;
}

void* vmt_state_device_ptr(const vmt_state* st) { return st ? st->d_states : nullptr; }

int vmt_device_status(int reset)
{
    const int v = vmt::read_generate_timeout(reset != 0);
    if (v < 0) return fail(VMT_ECUDA, "could not read the device status flag");
    if (v) return fail(VMT_ETIMEOUT, "a generation kernel gave up waiting for a bulk copy");
    return VMT_OK;
}

void vmt_free(vmt_state* st)
{
    if (!st) return;
    if (st->async_alloc) {
        // stream-ordered memory released without a stream: wait for the device
        if (st->d_states || st->d_pos) cudaDeviceSynchronize();
        if (st->d_states) cudaFreeAsync(st->d_states, nullptr);
        if (st->d_pos) cudaFreeAsync(st->d_pos, nullptr);
    } else {
        if (st->d_states) cudaFree(st->d_states);
        if (st->d_pos) cudaFree(st->d_pos);
    }
    if (st->units_free) cudaEventSynchronize(st->units_free), cudaEventDestroy(st->units_free);
    if (st->h_units) cudaFreeHost(st->h_units);
    if (st->d_units) cudaFree(st->d_units);
    if (st->d_counter) cudaFree(st->d_counter);
    delete st;
}

int vmt_tune_set(int variant, int lanes, int threads)
{
    if (!valid_variant(variant) || !valid_lanes(lanes)) return fail(VMT_EINVAL, "bad variant or lanes");
    const int idx = threads == 0 ? 0 : phase_index(variant, lanes, threads);
    if (idx < 0) return fail(VMT_EINVAL, "no kernel compiled with that CTA size for this variant and lane count");
    std::lock_guard<std::mutex> lk(g_tune_lock);
    read_tune_env_locked();
    g_tune_kcfg[variant][lanes] = idx;
    return VMT_OK;
}

int vmt_tune_get(int variant, int lanes)
{
    if (!valid_variant(variant) || !valid_lanes(lanes)) return fail(VMT_EINVAL, "bad variant or lanes");
    const vmt::KernelCfg* c = vmt::kernel_cfg(variant, lanes, vmt::tuned_kcfg(variant, lanes));
    return c ? c->threads : 0;
}

int vmt_tune_pass_cut(int variant, int lanes, int index, int* out8)
{
    if (!valid_variant(variant) || variant == VMT_SFMT19937 || !valid_lanes(lanes) || !out8)
        return fail(VMT_EINVAL, "bad argument");
    if (vmt::pass_cut(variant, lanes, index, out8) != 0)
        return fail(VMT_EINVAL, "no phase-form configuration with that index");
    return VMT_OK;
}

int vmt_tune_kernels(int variant, int lanes, int* desc, int cap)
{
    if (!valid_variant(variant) || !valid_lanes(lanes) || cap < 0 || (cap > 0 && !desc))
        return fail(VMT_EINVAL, "bad variant, lanes or buffer");
    const int n = vmt::kernel_cfg_count(variant, lanes);
    for (int i = 0; i < n && i < cap; ++i) {
        const vmt::KernelCfg* c = vmt::kernel_cfg(variant, lanes, i);
        desc[4 * i + 0] = c->form;
        desc[4 * i + 1] = c->lpc;
        desc[4 * i + 2] = c->threads;
        desc[4 * i + 3] = c->store;
    }
    return n;
}

int vmt_tune_set_kernel(int variant, int lanes, int index)
{
    if (!valid_variant(variant) || !valid_lanes(lanes)) return fail(VMT_EINVAL, "bad variant or lanes");
    const int n = vmt::kernel_cfg_count(variant, lanes);
    if (index < 0 || (index > 0 && index >= n)) return fail(VMT_EINVAL, "no compiled kernel configuration with that index");
    std::lock_guard<std::mutex> lk(g_tune_lock);
    read_tune_env_locked();
    g_tune_kcfg[variant][lanes] = index;
    return VMT_OK;
}

int vmt_tune_get_kernel(int variant, int lanes)
{
    if (!valid_variant(variant) || !valid_lanes(lanes)) return fail(VMT_EINVAL, "bad variant or lanes");
    return vmt::tuned_kcfg(variant, lanes);
}

int vmt_tune_save(const char* path)
{
    if (!path) return fail(VMT_EINVAL, "null path");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(VMT_EINVAL, std::string("cannot write ") + path);
    {
        std::lock_guard<std::mutex> lk(g_tune_lock);
        read_tune_env_locked();
        std::fprintf(f, "# variant lanes form lanes_per_cta threads store_bytes\n");
        for (int v = 0; v < 3; ++v)
            for (int m = 1; m <= 16; m *= 2)
                if (g_tune_kcfg[v][m]) {
                    const vmt::KernelCfg* c = vmt::kernel_cfg(v, m, g_tune_kcfg[v][m]);
                    if (c) std::fprintf(f, "%d %d %d %d %d %d\n", v, m, c->form, c->lpc, c->threads, c->store);
                }
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? VMT_OK : fail(VMT_EINVAL, std::string("cannot write ") + path);
}

int vmt_tune_load(const char* path)
{
    if (!path) return fail(VMT_EINVAL, "null path");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(VMT_EINVAL, std::string("cannot read ") + path);
    char line[160];
    int bad = 0;
    while (std::fgets(line, sizeof(line), f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int v = -1, m = 0, form = -1, lpc = 0, t = -1, store = 0;
        const int k = std::sscanf(line, "%d %d %d %d %d %d", &v, &m, &form, &lpc, &t, &store);
        if (k == 3) {   // "variant lanes threads": a phase-form CTA size
            if (vmt_tune_set(v, m, form) != VMT_OK) ++bad;
        } else if (k == 6 && valid_variant(v) && valid_lanes(m)) {
            int idx = -1;
            for (int i = 0; i < vmt::kernel_cfg_count(v, m); ++i) {
                const vmt::KernelCfg* c = vmt::kernel_cfg(v, m, i);
                if (c->form == form && c->lpc == lpc && c->threads == t && c->store == store) idx = i;
            }
            if (idx < 0 || vmt_tune_set_kernel(v, m, idx) != VMT_OK) ++bad;
        } else {
            ++bad;
        }
    }
    std::fclose(f);
    return bad ? fail(VMT_EINVAL, "tuning file has entries that match no compiled kernel") : VMT_OK;
}

int vmt_autotune_grid(int variant, int lanes, int64_t count, int nseg, const int64_t* counts, const int* dtypes,
                      int reps, void* cuda_stream, double* ms_out, int cap, int* best_index)
{
    if (!valid_variant(variant) || !valid_lanes(lanes) || count < 1 || reps < 1 || nseg < 1 || nseg > VMT_MAXSEG ||
        !counts || !dtypes || cap < 0 || (cap > 0 && !ms_out))
        return fail(VMT_EINVAL, "bad autotune arguments");
    for (int i = 0; i < nseg; ++i)
        if (counts[i] < 1 || dtypes[i] < VMT_U32 || dtypes[i] > VMT_F64) return fail(VMT_EINVAL, "bad autotune segment");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int ncand = std::max(1, vmt::kernel_cfg_count(variant, lanes));
    std::vector<uint64_t> seeds(static_cast<size_t>(count));
    for (int64_t g = 0; g < count; ++g) seeds[static_cast<size_t>(g)] = 0x9E3779B97F4A7C15ull * static_cast<uint64_t>(g + 1);
    vmt_state* st = nullptr;
    int rc = vmt_init_batch(&st, variant, lanes, count, seeds.data(), nullptr, cuda_stream);
    if (rc) return rc;
    std::vector<void*> outs(static_cast<size_t>(nseg), nullptr);
    for (int i = 0; i < nseg; ++i)
        if (cudaMalloc(&outs[static_cast<size_t>(i)], static_cast<size_t>(count * counts[i] * elem_bytes(dtypes[i]))) !=
            cudaSuccess) {
            cudaGetLastError();
            for (void* o : outs)
                if (o) cudaFree(o);
            vmt_free(st);
            return fail(VMT_ENOMEM, "autotune output buffer");
        }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int prev = vmt::tuned_kcfg(variant, lanes);
    // two alternating rounds over the candidates, each candidate's time the
    // mean of `reps` calls after a warm-up; a candidate keeps its better round
    std::vector<double> t_best(static_cast<size_t>(ncand), 1e30);
    for (int round = 0; round < 2 && rc == VMT_OK; ++round)
        for (int k = 0; k < ncand && rc == VMT_OK; ++k) {
            {
                std::lock_guard<std::mutex> lk(g_tune_lock);
                g_tune_kcfg[variant][lanes] = k;
            }
            rc = vmt_generate_multi(st, nseg, counts, dtypes, outs.data(), cuda_stream);   // warm-up
            if (rc) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == VMT_OK; ++r)
                rc = vmt_generate_multi(st, nseg, counts, dtypes, outs.data(), cuda_stream);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            t_best[static_cast<size_t>(k)] = std::min(t_best[static_cast<size_t>(k)], static_cast<double>(ms) / reps);
        }
    int best = 0;
    for (int k = 1; k < ncand; ++k)
        if (t_best[static_cast<size_t>(k)] < t_best[static_cast<size_t>(best)]) best = k;
    {
        std::lock_guard<std::mutex> lk(g_tune_lock);
        g_tune_kcfg[variant][lanes] = rc == VMT_OK ? best : prev;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (void* o : outs) cudaFree(o);
    vmt_free(st);
    if (rc) return rc;
    for (int k = 0; k < ncand && k < cap; ++k) ms_out[k] = t_best[static_cast<size_t>(k)];
    if (best_index) *best_index = best;
    return VMT_OK;
}

int vmt_autotune_multi(int variant, int lanes, int64_t count, int nseg, const int64_t* counts, const int* dtypes,
                       int reps, void* cuda_stream, int* best_threads, double* best_ms)
{
    double ms[64];
    int best = 0;
    const int rc = vmt_autotune_grid(variant, lanes, count, nseg, counts, dtypes, reps, cuda_stream, ms, 64, &best);
    if (rc) return rc;
    const vmt::KernelCfg* c = vmt::kernel_cfg(variant, lanes, best);
    if (best_threads) *best_threads = c ? c->threads : 0;
    if (best_ms) *best_ms = ms[best];
    return VMT_OK;
}

int vmt_autotune(int variant, int lanes, int64_t count, int64_t n_per_gen, int dtype, int reps, void* cuda_stream,
                 int* best_threads, double* best_ms)
{
    return vmt_autotune_multi(variant, lanes, count, 1, &n_per_gen, &dtype, reps, cuda_stream, best_threads, best_ms);
}

int vmt_poly_minpoly(const uint64_t* bits, int64_t n, uint64_t* mu_out, int64_t cap_words)
{
    if (!bits || !mu_out || n < 1) return fail(VMT_EINVAL, "bad argument");
    Poly mu = vmt::gf2::berlekamp_massey(bits, n);
    const int d = vmt::gf2::degree(mu);
    const int64_t nw = d / 64 + 1;
    if (cap_words < nw) return fail(VMT_EINVAL, "mu_out too small");
    std::memset(mu_out, 0, static_cast<size_t>(cap_words) * 8);
    std::memcpy(mu_out, mu.data(), static_cast<size_t>(nw) * 8);
    return d;
}

int vmt_poly_mulmod(const uint64_t* a, const uint64_t* b, const uint64_t* mu, uint64_t* out, int64_t nw)
{
    if (!a || !b || !mu || !out || nw < 1) return fail(VMT_EINVAL, "bad argument");
    try {
        vmt::gf2::Modulus m(Poly(mu, mu + nw));
        Poly r = m.mul(Poly(a, a + nw), Poly(b, b + nw));
        std::memset(out, 0, static_cast<size_t>(nw) * 8);
        std::memcpy(out, r.data(), std::min<size_t>(r.size(), static_cast<size_t>(nw)) * 8);
    } catch (const std::exception& e) {
        return fail(VMT_EINVAL, e.what());
    }
    return VMT_OK;
}

int vmt_poly_x2pow(const uint64_t* mu, int64_t nw, int q_lo, int q_hi, uint64_t* out)
{
    if (!mu || !out || nw < 1 || q_lo < 0 || q_hi < q_lo) return fail(VMT_EINVAL, "bad argument");
    try {
        vmt::gf2::Modulus m(Poly(mu, mu + nw));
        Poly r = m.x_pow_2q(0);
        for (int q = 0; q <= q_hi; ++q) {
            if (q >= q_lo) {
                uint64_t* dst = out + static_cast<int64_t>(q - q_lo) * nw;
                std::memset(dst, 0, static_cast<size_t>(nw) * 8);
                std::memcpy(dst, r.data(), std::min<size_t>(r.size(), static_cast<size_t>(nw)) * 8);
            }
            if (q < q_hi) r = m.sqr(r);
        }
    } catch (const std::exception& e) {
        return fail(VMT_EINVAL, e.what());
    }
    return VMT_OK;
}

}  // extern "C"
