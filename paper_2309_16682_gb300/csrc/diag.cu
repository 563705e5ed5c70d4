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

#include "bulk.cuh"
#include "vmt_internal.hpp"

namespace {

// Waits, with the bounded wait of the generation kernels, on an mbarrier
// that nothing arrives at; records whether the wait gave up and how long it
// took.  Used to check that a stalled wait ends with a status, not a hang.
__global__ void wait_selftest_kernel(unsigned long long limit_ns, int* gave_up, unsigned long long* elapsed_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        vmt::dev::mbar_init(&bar, 1);
        vmt::dev::fence_mbar_init();
    }
    __syncthreads();
    const unsigned long long t0 = vmt::dev::globaltimer_ns();
    const bool done = vmt::dev::mbar_wait(&bar, 0u, limit_ns);
    const unsigned long long t1 = vmt::dev::globaltimer_ns();
    __syncthreads();
    if (threadIdx.x == 0) {
        *gave_up = done ? 0 : 1;
        *elapsed_ns = t1 - t0;
        vmt::dev::mbar_inval(&bar);
    }
}

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

extern "C" int vmt_selftest_wait(int64_t limit_ns, int64_t* elapsed_ns)
{
    if (limit_ns < 1000 || limit_ns > 10000000000LL) {
        vmt::set_last_error("vmt_selftest_wait: limit must be in 1 us .. 10 s");
        return VMT_EINVAL;
    }
    int* d_flag = nullptr;
    unsigned long long* d_el = nullptr;
    if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess || cudaMalloc(&d_el, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (d_flag) cudaFree(d_flag);
        vmt::set_last_error("vmt_selftest_wait: allocation failed");
        return VMT_ENOMEM;
    }
    wait_selftest_kernel<<<1, 32>>>(static_cast<unsigned long long>(limit_ns), d_flag, d_el);
    int flag = 0;
    unsigned long long el = 0;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&el, d_el, sizeof(el), cudaMemcpyDeviceToHost);
    cudaFree(d_flag);
    cudaFree(d_el);
    if (e != cudaSuccess) {
        vmt::set_last_error((std::string("vmt_selftest_wait: ") + cudaGetErrorString(e)).c_str());
        return VMT_ECUDA;
    }
    if (elapsed_ns) *elapsed_ns = static_cast<int64_t>(el);
    return flag ? VMT_ETIMEOUT : VMT_OK;
}
