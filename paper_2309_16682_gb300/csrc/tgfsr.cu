// tgfsr.cu -- twisted GFSR generators with run-time parameters (C ABI).
//
// The V-family construction of Sec. 3 needs three things from its base
// generator: the recurrence (eq. step), a linear output function (eq.
// tempering) and the jump c(F) X with c = x^J mod the minimal polynomial
// (Sec. 3.1).  None of them is specific to the parameters of MT19937, so this
// file offers them for any twisted GFSR of that shape: w-bit words (w <= 32),
// n words of state (one of the compiled sizes), middle distance m, separation
// point r and twist constant a, with an optional tempering of the MT form.
// The jump runs the window-correlation kernels of jump.cu (the same templates
// as the MT19937 and SFMT19937 jumps, with the sequence extended by this
// recurrence); the minimal polynomial and x^J come from the host polynomial
// helpers (vmt_poly_*) applied to output bits.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "vmt_internal.hpp"

namespace {

constexpr int kGenThreads = 128;
constexpr int kMaxN = 17;

struct TgDev {
    int n, m;
    uint32_t upper, lower, a, wmask;
    int temper;
    int u, s, t, l;
    uint32_t d, b, c;
};

__device__ __forceinline__ uint32_t tg_step(uint32_t xk, uint32_t xk1, uint32_t xkm, const TgDev& g)
{
    const uint32_t y = (xk & g.upper) | (xk1 & g.lower);
    return xkm ^ (y >> 1) ^ ((y & 1u) ? g.a : 0u);
}

__device__ __forceinline__ uint32_t tg_out(uint32_t y, const TgDev& g)
{
    if (!g.temper) return y;
    y ^= (y >> g.u) & g.d;
    y ^= (y << g.s) & g.b;
    y ^= (y << g.t) & g.c;
    y ^= y >> g.l;
    return y & g.wmask;
}

// One thread per state: the window of n words in shared memory (word j of
// thread t at ring[j * kGenThreads + t], a circular buffer), k-th output word
// of state i = (generator gi, lane t) stored at out[(gi * n_out + k) * lanes + t]
// (the interleaved order S[kM + t] of eq. combseq), the advanced window
// written back oldest word first.
__global__ void __launch_bounds__(kGenThreads) tgfsr_generate_kernel(TgDev g, long long count, int lanes,
                                                                     uint32_t* states, long long n_out, uint32_t* out)
{
    __shared__ uint32_t ring[kMaxN * kGenThreads];
    const int tid = threadIdx.x;
    const long long i = static_cast<long long>(blockIdx.x) * kGenThreads + tid;
    if (i >= count) return;
    const int n = g.n;
    uint32_t* st = states + i * n;
    for (int j = 0; j < n; ++j) ring[j * kGenThreads + tid] = st[j];
    const long long gi = i / lanes;
    const int t = static_cast<int>(i % lanes);
    uint32_t* o = out + gi * n_out * lanes + t;
    int p = 0;   // ring slot of the oldest word x_k
    for (long long k = 0; k < n_out; ++k) {
        const int p1 = p + 1 == n ? 0 : p + 1;
        const int pm = p + g.m >= n ? p + g.m - n : p + g.m;
        const uint32_t x = tg_step(ring[p * kGenThreads + tid], ring[p1 * kGenThreads + tid],
                                   ring[pm * kGenThreads + tid], g);
        ring[p * kGenThreads + tid] = x;   // x_{k+n} takes the slot of x_k
        o[k * lanes] = tg_out(x, g);
        p = p1;
    }
    for (int j = 0; j < n; ++j) {
        const int q = p + j >= n ? p + j - n : p + j;
        st[j] = ring[q * kGenThreads + tid];
    }
}

int fail_tg(int code, const std::string& msg)
{
    vmt::set_last_error(msg.c_str());
    return code;
}

bool compiled_n(int n)
{
    for (int c : vmt::kTgfsrSizes)
        if (c == n) return true;
    return false;
}

int check_params(const vmt_tgfsr* g, TgDev* d)
{
    if (!g) return fail_tg(VMT_EINVAL, "vmt_tgfsr: null parameters");
    if (g->w < 2 || g->w > 32) return fail_tg(VMT_EINVAL, "vmt_tgfsr: w must be in 2..32");
    if (!compiled_n(g->n)) return fail_tg(VMT_EINVAL, "vmt_tgfsr: n is not one of the compiled sizes (4, 5, 17)");
    if (g->m < 1 || g->m >= g->n) return fail_tg(VMT_EINVAL, "vmt_tgfsr: m must be in 1..n-1");
    if (g->r < 1 || g->r >= g->w) return fail_tg(VMT_EINVAL, "vmt_tgfsr: r must be in 1..w-1");
    const uint32_t wmask = g->w == 32 ? 0xFFFFFFFFu : ((1u << g->w) - 1u);
    if (g->a & ~wmask) return fail_tg(VMT_EINVAL, "vmt_tgfsr: a has bits above w");
    if (g->temper && (g->u < 0 || g->u >= g->w || g->s < 0 || g->s >= g->w || g->t < 0 || g->t >= g->w ||
                      g->l < 0 || g->l >= g->w))
        return fail_tg(VMT_EINVAL, "vmt_tgfsr: tempering shifts must be in 0..w-1");
    d->n = g->n;
    d->m = g->m;
    d->lower = (1u << g->r) - 1u;
    d->upper = wmask ^ d->lower;
    d->a = g->a;
    d->wmask = wmask;
    d->temper = g->temper ? 1 : 0;
    d->u = g->u;
    d->s = g->s;
    d->t = g->t;
    d->l = g->l;
    d->d = g->d;
    d->b = g->b;
    d->c = g->c;
    return VMT_OK;
}

}  // namespace

extern "C" {

int vmt_tgfsr_jump(const vmt_tgfsr* g, int64_t count, void* states, const uint64_t* poly, int64_t nbits, int kernel,
                   void* cuda_stream)
{
    TgDev d{};
    int rc = check_params(g, &d);
    if (rc) return rc;
    if (count < 0 || (count > 0 && (!states || !poly))) return fail_tg(VMT_EINVAL, "vmt_tgfsr_jump: bad states or poly");
    if (nbits < 0 || nbits > 32LL * vmt::kPolyWords - 64) return fail_tg(VMT_EINVAL, "vmt_tgfsr_jump: nbits must be in 0..20416");
    if (kernel != 0 && kernel != 1) return fail_tg(VMT_EINVAL, "vmt_tgfsr_jump: kernel must be 0 (warp) or 1 (CTA)");
    if (count == 0) return VMT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // the polynomial row (bits at and above nbits cleared) and one item per state
    std::vector<uint32_t> row(vmt::kPolyWords, 0u);
    const int64_t nw = (nbits + 63) / 64;
    std::memcpy(row.data(), poly, static_cast<size_t>(nw) * 8);
    if (nbits % 64) {
        uint64_t last = 0;
        std::memcpy(&last, row.data() + 2 * (nw - 1), 8);
        last &= (1ull << (nbits % 64)) - 1ull;
        std::memcpy(row.data() + 2 * (nw - 1), &last, 8);
    }
    int deg = -1;
    for (int w = vmt::kPolyWords - 1; w >= 0 && deg < 0; --w)
        if (row[static_cast<size_t>(w)]) deg = 32 * w + 31 - __builtin_clz(row[static_cast<size_t>(w)]);
    std::vector<vmt::JumpItem> items(static_cast<size_t>(count));
    for (int64_t i = 0; i < count; ++i) {
        vmt::JumpItem& it = items[static_cast<size_t>(i)];
        it.src = static_cast<uint32_t*>(states) + i * g->n;
        it.dst = static_cast<uint32_t*>(states) + i * g->n;
        it.src_stride = 1;
        it.dst_stride = 1;
        it.poly = 0;
        it.deg = deg;
    }
    uint32_t* d_row = nullptr;
    vmt::JumpItem* d_items = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&d_row), row.size() * 4, s) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void**>(&d_items), items.size() * sizeof(vmt::JumpItem), s) != cudaSuccess) {
        cudaGetLastError();
        if (d_row) cudaFreeAsync(d_row, s);
        return fail_tg(VMT_ENOMEM, "vmt_tgfsr_jump: scratch allocation failed");
    }
    // pageable sources: each copy has read its source when it returns
    cudaError_t e = cudaMemcpyAsync(d_row, row.data(), row.size() * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(vmt::JumpItem), cudaMemcpyHostToDevice, s);
    vmt::JumpGrid gr{};
    gr.tg_m = static_cast<unsigned>(d.m);
    gr.tg_upper = d.upper;
    gr.tg_lower = d.lower;
    gr.tg_a = d.a;
    if (e == cudaSuccess) e = vmt::launch_tgfsr_jump(g->n, kernel == 1, d_items, count, gr, d_row, s);
    cudaFreeAsync(d_items, s);
    cudaFreeAsync(d_row, s);
    if (e != cudaSuccess) return fail_tg(VMT_ECUDA, std::string("vmt_tgfsr_jump: ") + cudaGetErrorString(e));
    return VMT_OK;
}

int vmt_tgfsr_generate(const vmt_tgfsr* g, int64_t count, int lanes, void* states, int64_t n, void* out,
                       void* cuda_stream)
{
    TgDev d{};
    int rc = check_params(g, &d);
    if (rc) return rc;
    if (count < 0 || lanes < 1 || count % lanes != 0 || n < 0)
        return fail_tg(VMT_EINVAL, "vmt_tgfsr_generate: count must be a multiple of lanes >= 1, n >= 0");
    if (count == 0) return VMT_OK;
    if (!states || (n > 0 && !out)) return fail_tg(VMT_EINVAL, "vmt_tgfsr_generate: null states or output");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long grid = (count + kGenThreads - 1) / kGenThreads;
    tgfsr_generate_kernel<<<static_cast<unsigned>(grid), kGenThreads, 0, s>>>(
        d, count, lanes, static_cast<uint32_t*>(states), n, static_cast<uint32_t*>(out));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_tg(VMT_ECUDA, std::string("vmt_tgfsr_generate: ") + cudaGetErrorString(e));
    return VMT_OK;
}

}  // extern "C"
