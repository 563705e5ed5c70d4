// scalar.cu -- buffered scalar queries (the paper's scalar query mode served
// from a buffer: state recurrence and tempering run in bulk and single
// outputs are read from a small buffer, Sec. 4.4.1 "Scalar Performance and
// Optimized Buffering").
//
// Here the bulk step is a GPU generation of K outputs of one V-generator
// written straight into pinned host memory (mapped into the GPU's address
// space).  Two host halves alternate: while the host reads one, the GPU
// refills the other on the object's own stream, so a query is a bounds check
// and a load except once every K queries, when it waits for the refill that
// was started K queries earlier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>

#include "vmt_internal.hpp"

struct vmt_scalar {
    vmt_state* st = nullptr;
    int dtype = VMT_U32;
    int esize = 4;
    int64_t K = 0;               // outputs per half
    cudaStream_t s = nullptr;
    unsigned char* host[2] = {nullptr, nullptr};   // pinned halves
    void* mapped[2] = {nullptr, nullptr};          // the same halves as device addresses
    cudaEvent_t ready[2] = {nullptr, nullptr};
    int cur = 0;                 // half being read
    int64_t pos = 0;             // next output in it
};

namespace {

// start refilling half h: the kernels write K outputs into it directly
int refill(vmt_scalar* q, int h)
{
    int rc = vmt_generate(q->st, q->K, q->dtype, q->mapped[h], q->s);
    if (rc) return rc;
    if (cudaEventRecord(q->ready[h], q->s) != cudaSuccess) {
        vmt::set_last_error("vmt_scalar: refill failed");
        return VMT_ECUDA;
    }
    return VMT_OK;
}

// the current half is used up: wait for the other one and refill this one
inline int advance(vmt_scalar* q)
{
    const int other = q->cur ^ 1;
    if (cudaEventSynchronize(q->ready[other]) != cudaSuccess) {
        vmt::set_last_error("vmt_scalar: waiting for a refill failed");
        return VMT_ECUDA;
    }
    const int used = q->cur;
    q->cur = other;
    q->pos = 0;
    return refill(q, used);
}

}  // namespace

extern "C" {

int vmt_scalar_create(vmt_scalar** out, int variant, int lanes, uint64_t seed, uint64_t jump, int dtype,
                      int64_t buffer_outputs)
{
    if (!out) {
        vmt::set_last_error("vmt_scalar_create: null handle");
        return VMT_EINVAL;
    }
    *out = nullptr;
    if (buffer_outputs < 1024 || buffer_outputs > (int64_t(1) << 28)) {
        vmt::set_last_error("vmt_scalar_create: buffer_outputs must be in 1024 .. 2^28");
        return VMT_EINVAL;
    }
    std::unique_ptr<vmt_scalar> q(new vmt_scalar());
    q->dtype = dtype;
    q->esize = (dtype == VMT_U32 || dtype == VMT_F32) ? 4 : 8;
    q->K = buffer_outputs;
    if (cudaStreamCreateWithFlags(&q->s, cudaStreamNonBlocking) != cudaSuccess) {
        vmt::set_last_error("vmt_scalar_create: stream creation failed");
        return VMT_ECUDA;
    }
    int rc = vmt_init(&q->st, variant, lanes, seed, jump, q->s);
    bool ok = rc == VMT_OK;
    for (int h = 0; h < 2 && ok; ++h)
        ok = cudaHostAlloc(reinterpret_cast<void**>(&q->host[h]), static_cast<size_t>(q->K * q->esize),
                           cudaHostAllocMapped) == cudaSuccess &&
             cudaHostGetDevicePointer(&q->mapped[h], q->host[h], 0) == cudaSuccess &&
             cudaEventCreateWithFlags(&q->ready[h], cudaEventDisableTiming) == cudaSuccess;
    if (ok) rc = refill(q.get(), 0);
    if (ok && !rc) rc = refill(q.get(), 1);
    if (ok && !rc && cudaEventSynchronize(q->ready[0]) != cudaSuccess) rc = VMT_ECUDA;
    if (!ok || rc) {
        if (!rc) {
            cudaGetLastError();
            vmt::set_last_error("vmt_scalar_create: allocation failed");
            rc = VMT_ENOMEM;
        }
        vmt_scalar_destroy(q.release());
        return rc;
    }
    *out = q.release();
    return VMT_OK;
}

int vmt_scalar_next(vmt_scalar* q, void* value)
{
    if (!q || !value) return VMT_EINVAL;
    if (q->pos == q->K) {
        const int rc = advance(q);
        if (rc) return rc;
    }
    std::memcpy(value, q->host[q->cur] + q->pos * q->esize, static_cast<size_t>(q->esize));
    ++q->pos;
    return VMT_OK;
}

int vmt_scalar_take(vmt_scalar* q, int64_t n, void* out_host)
{
    if (!q || n < 0 || (n > 0 && !out_host)) return VMT_EINVAL;
    unsigned char* dst = static_cast<unsigned char*>(out_host);
    while (n > 0) {
        if (q->pos == q->K) {
            const int rc = advance(q);
            if (rc) return rc;
        }
        const int64_t k = std::min<int64_t>(n, q->K - q->pos);
        std::memcpy(dst, q->host[q->cur] + q->pos * q->esize, static_cast<size_t>(k * q->esize));
        q->pos += k;
        dst += k * q->esize;
        n -= k;
    }
    return VMT_OK;
}

int vmt_scalar_drain(vmt_scalar* q, int64_t count, uint64_t* checksum)
{
    if (!q || count < 0 || !checksum) return VMT_EINVAL;
    uint64_t acc = 0;
    if (q->esize == 4) {
        for (int64_t i = 0; i < count; ++i) {
            uint32_t v;
            const int rc = vmt_scalar_next(q, &v);
            if (rc) return rc;
            acc = (acc ^ v) * 0x100000001B3ull;
        }
    } else {
        for (int64_t i = 0; i < count; ++i) {
            uint64_t v;
            const int rc = vmt_scalar_next(q, &v);
            if (rc) return rc;
            acc = (acc ^ v) * 0x100000001B3ull;
        }
    }
    *checksum = acc;
    return VMT_OK;
}

void vmt_scalar_destroy(vmt_scalar* q)
{
    if (!q) return;
    if (q->s) cudaStreamSynchronize(q->s);
    for (int h = 0; h < 2; ++h) {
        if (q->host[h]) cudaFreeHost(q->host[h]);
        if (q->ready[h]) cudaEventDestroy(q->ready[h]);
    }
    if (q->st) vmt_free(q->st);
    if (q->s) cudaStreamDestroy(q->s);
    delete q;
}

}  // extern "C"
