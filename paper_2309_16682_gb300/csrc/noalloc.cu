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
// device current, looks the address up with cudaGetSymbolAddress and keeps it.
// That first call should come before any stream capture.  All calls share the
// one array, which keeps the previous call's contents: the polynomial row is
// cleared past the caller's words on every call, and calls that overlap on the
// GPU race on the array.
#include <mutex>

#include "vmt_device.cuh"
#include "vmt_internal.hpp"

namespace {

constexpr long long kMaxLaneStates = VMT_NOALLOC_MAX_LANE_STATES;
constexpr size_t kPolyBytes = sizeof(uint32_t) * vmt::kPolyWords;
constexpr size_t kItemBytes = sizeof(vmt::JumpItem) * kMaxLaneStates;
constexpr size_t kScratchBytes = kPolyBytes + kItemBytes;   // polynomial row, then the items

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
void* g_scratch_ptr[kMaxDevices] = {};

int fail_static(int code, const char* msg)
{
    vmt::set_last_error(msg);
    return code;
}

// item i = lane t of generator g, jumped in place
__global__ void fill_lane_items(vmt::JumpItem* items, char* states, long long count, int lanes, long long gen_bytes,
                                int unit_bytes, int deg)
{
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
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
    if (nbits < 0 || nbits > 32LL * vmt::kPolyWords - 64)
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
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail_static(VMT_ECUDA, "vmt_jump_noalloc: cudaGetSymbolAddress failed");
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    uint32_t* row = static_cast<uint32_t*>(scratch);
    vmt::JumpItem* items = reinterpret_cast<vmt::JumpItem*>(static_cast<char*>(scratch) + kPolyBytes);

    // polynomial row: the caller's words (little-endian uint64 = two uint32),
    // the bits at and above nbits cleared, the rest of the row zeroed
    const int64_t full = nbits / 64;
    const int rem = static_cast<int>(nbits % 64);
    int deg = -1;
    for (int64_t w = (rem ? full : full - 1); w >= 0 && deg < 0; --w) {
        uint64_t v = poly[w];
        if (w == full) v &= (1ull << rem) - 1ull;
        if (v) deg = static_cast<int>(64 * w + 63 - __builtin_clzll(v));
    }
    cudaError_t e = cudaMemsetAsync(row, 0, kPolyBytes, s);
    if (e == cudaSuccess && full > 0) e = cudaMemcpyAsync(row, poly, static_cast<size_t>(full) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && rem) {
        const uint64_t last = poly[full] & ((1ull << rem) - 1ull);
        e = cudaMemcpyAsync(row + 2 * full, &last, 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // `last` lives on this stack frame
    }
    if (e != cudaSuccess) return fail_static(VMT_ECUDA, "vmt_jump_noalloc: copying the polynomial failed");

    const long long n = count * lanes;
    const int unit_bytes = vmt::word_bytes(variant) * vmt::words_per_unit(variant);
    const long long gen_bytes = vmt::state_bytes_per_gen(variant, lanes);
    fill_lane_items<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
        items, static_cast<char*>(vmt_state_device_ptr(st)), count, lanes, gen_bytes, unit_bytes, deg);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = vmt::launch_jump(variant, items, n, row, s);
    if (e != cudaSuccess) return fail_static(VMT_ECUDA, "vmt_jump_noalloc: kernel launch failed");
    return VMT_OK;
}
