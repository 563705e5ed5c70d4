// noalloc.cu -- vmt_jump_noalloc: the jump of vmt_jump without any allocation.
//
// vmt_jump allocates two pieces of device scratch per call: the polynomial
// row and the table of lane-jump work items that the jump kernel reads.
// Callers that cannot allocate device memory -- code that runs while a
// framework's caching allocator owns all free HBM, real-time loops that must
// not pay for cudaMalloc/cudaFree, or plug-ins whose host application forbids
// library allocations -- use this entry point instead.  Its scratch is the
// file-scope array below, sized for the largest call it accepts; every GPU
// that loads the library holds that array until the process exits.
//
// The host cannot use the array's name as a device address (in host code the
// name is a host-side stand-in), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and keeps it,
// together with the unique id of the CUDA context it belongs to; a later call
// in another context of that device (after cudaDeviceReset) looks it up again.
// That first call should come before any stream capture.  All calls share the
// one array, which keeps the previous call's contents: every call rewrites the
// whole polynomial row and every work item it uses, and calls that overlap on
// the GPU race on the array.
//
// The caller's polynomial reaches the GPU as a kernel parameter (at most 2560
// bytes), which the launch copies: the host buffer is read before the call
// returns, whatever kind of memory it is, and no copy or stream
// synchronisation is issued.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "vmt_device.cuh"
#include "vmt_internal.hpp"

namespace {

constexpr long long kMaxLaneStates = VMT_NOALLOC_MAX_LANE_STATES;
constexpr size_t kPolyBytes = sizeof(uint32_t) * vmt::kPolyWords;
constexpr size_t kItemBytes = sizeof(vmt::JumpItem) * kMaxLaneStates;
constexpr size_t kScratchBytes = kPolyBytes + kItemBytes;   // polynomial row, then the items
constexpr int kMaxNbits = 32 * vmt::kPolyWords - 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// the polynomial row by value: kPolyWords u32 words, bits at and above nbits
// already cleared on the host
struct PolyRow {
    uint32_t w[vmt::kPolyWords];
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
struct DeviceScratch {
    void* ptr = nullptr;
    unsigned long long ctx_id = 0;
};
DeviceScratch g_scratch[kMaxDevices];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_entry_points_tried = false;

int fail_static(int code, const char* msg)
{
    vmt::set_last_error(msg);
    return code;
}

// unique id of the current context (0 when it cannot be told): the primary
// context of `dev` is made current first, as every runtime call on it does
unsigned long long current_context_id(int dev)
{
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        cudaDriverEntryPointQueryResult q{};
        void* f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    if (cudaSetDevice(dev) != cudaSuccess) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Writes the whole polynomial row (every call: the array keeps the previous
// call's row) and item i = lane t of generator g, jumped in place.
__global__ void noalloc_prepare(PolyRow p, uint32_t* row, vmt::JumpItem* items, char* states, long long count,
                                int lanes, long long gen_bytes, int unit_bytes, int deg)
{
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < vmt::kPolyWords) row[i] = p.w[i];
    if (i >= count * lanes) return;
    const long long g = i / lanes;
    const int t = static_cast<int>(i % lanes);
    vmt::JumpItem it;
    it.src = states + g * gen_bytes + static_cast<long long>(t) * unit_bytes;
    it.dst = states + g * gen_bytes + static_cast<long long>(t) * unit_bytes;
    it.src_stride = lanes;
    it.dst_stride = lanes;
    it.poly = 0;
    it.deg = deg;
    items[i] = it;
}

}  // namespace

extern "C" int vmt_jump_noalloc(vmt_state* st, const uint64_t* poly, int64_t nbits, void* cuda_stream)
{
    if (!st || !poly) return fail_static(VMT_EINVAL, "vmt_jump_noalloc: null argument");
    int variant = 0, lanes = 0;
    int64_t count = 0, pos = 0;
    if (vmt_state_info(st, &variant, &lanes, &count, &pos) != VMT_OK)
        return fail_static(VMT_EINVAL, "vmt_jump_noalloc: bad state");
    if (nbits < 0 || nbits > kMaxNbits)
        return fail_static(VMT_EINVAL, "vmt_jump_noalloc: nbits must be in 0..20416");
    if (count * lanes > kMaxLaneStates)
        return fail_static(VMT_EINVAL,
                           "vmt_jump_noalloc: count * lanes exceeds the static scratch limit "
                           "VMT_NOALLOC_MAX_LANE_STATES (16384 lane-states)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail_static(VMT_ECUDA, "vmt_jump_noalloc: no usable current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_lock);
        const unsigned long long id = current_context_id(dev);
        DeviceScratch& ds = g_scratch[dev];
        if (!ds.ptr || (id != 0 && id != ds.ctx_id)) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail_static(VMT_ECUDA, "vmt_jump_noalloc: cudaGetSymbolAddress failed");
            ds.ptr = p;
            ds.ctx_id = id;
        }
        scratch = ds.ptr;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t* row = static_cast<uint32_t*>(scratch);
    vmt::JumpItem* items = reinterpret_cast<vmt::JumpItem*>(static_cast<char*>(scratch) + kPolyBytes);

    // the caller's words (little-endian uint64 = two uint32), the bits at and
    // above nbits cleared, the rest of the row zero
    PolyRow p;
    std::memset(&p, 0, sizeof(p));
    const int64_t nw = (nbits + 63) / 64;
    std::memcpy(p.w, poly, static_cast<size_t>(nw) * 8);
    const int rem = static_cast<int>(nbits % 64);
    if (rem) {
        uint64_t last = 0;
        std::memcpy(&last, p.w + 2 * (nw - 1), 8);
        last &= (1ull << rem) - 1ull;
        std::memcpy(p.w + 2 * (nw - 1), &last, 8);
    }
    int deg = -1;
    for (int w = vmt::kPolyWords - 1; w >= 0 && deg < 0; --w)
        if (p.w[w]) deg = 32 * w + 31 - __builtin_clz(p.w[w]);

    const long long n = count * lanes;
    const long long threads = n > vmt::kPolyWords ? n : vmt::kPolyWords;
    const int unit_bytes = vmt::word_bytes(variant) * vmt::words_per_unit(variant);
    const long long gen_bytes = vmt::state_bytes_per_gen(variant, lanes);
    noalloc_prepare<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, s>>>(
        p, row, items, static_cast<char*>(vmt_state_device_ptr(st)), count, lanes, gen_bytes, unit_bytes, deg);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = vmt::launch_jump(variant, items, n, row, s);
    if (e != cudaSuccess) return fail_static(VMT_ECUDA, "vmt_jump_noalloc: kernel launch failed");
    return VMT_OK;
}
