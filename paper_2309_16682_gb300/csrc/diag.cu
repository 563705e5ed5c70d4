// diag.cu -- device diagnostics.
//
// vmt_measure_store_bw: the HBM write ceiling that the generation kernels
// (which mostly write) are compared with, measured by a store-only kernel:
// 16-byte streaming stores over a buffer much larger than L2, best of `reps`
// launches.  Not a paper item; a measuring stick for the roofline.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>

#include "vmt_internal.hpp"

namespace {

__global__ void store_only_kernel(uint4* p, long long n16, uint32_t tag)
{
    const uint4 v = make_uint4(tag, tag ^ 0x9E3779B9u, tag + 1u, ~tag);
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n16;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        __stcs(p + i, v);
}

}  // namespace

extern "C" int vmt_measure_store_bw(int64_t bytes, int reps, double* best_gbs, void* cuda_stream)
{
    if (!best_gbs || bytes < (int64_t(1) << 20) || reps < 1) {
        vmt::set_last_error("vmt_measure_store_bw: need bytes >= 1 MiB, reps >= 1 and an output");
        return VMT_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const long long n16 = bytes / 16;
    void* buf = nullptr;
    if (cudaMallocAsync(&buf, static_cast<size_t>(n16) * 16, s) != cudaSuccess) {
        cudaGetLastError();
        vmt::set_last_error("vmt_measure_store_bw: allocation failed");
        return VMT_ENOMEM;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    // two launch shapes (a few large CTAs per SM, many small ones); best of all
    const int shapes[2][2] = {{4, 512}, {16, 256}};
    for (int r = 0; r < reps + 1; ++r)
        for (const auto& sh : shapes) {
            cudaEventRecord(e0, s);
            store_only_kernel<<<static_cast<unsigned>(sms * sh[0]), sh[1], 0, s>>>(static_cast<uint4*>(buf), n16,
                                                                                    static_cast<uint32_t>(r));
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0) best = std::min(best, ms);   // launch 0 of each shape is a warm-up
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(buf, s);
    const cudaError_t err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
        vmt::set_last_error((std::string("vmt_measure_store_bw: ") + cudaGetErrorString(err)).c_str());
        return VMT_ECUDA;
    }
    *best_gbs = static_cast<double>(n16) * 16.0 / (best * 1e-3) / 1e9;
    return VMT_OK;
}
