// sem_probe.cu -- device-fact probe: sustained FMA issue rate of the FP64 and
// FP32 pipes (flops/s), for the ALU roofline of the operator kernels.  Each
// thread runs 8 independent FMA chains so that latency is hidden; the grid
// fills every SM several times over.
#include <cuda_runtime.h>

#include "sem_internal.h"

namespace sem {

template <typename T>
__global__ void fma_probe_kernel(T *out, int iters, T a, T b) {
    T v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = T(threadIdx.x + q);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = fma(v[q], a, b);
    }
    T s = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) s += v[q];
    if (s == T(-12345.678)) out[0] = s;  // keeps the chains live; never true in practice
}

int probe_fma_rate(int dtype, int iters, double *flops_per_s) {
    if (iters < 1 || iters > (1 << 24)) return set_error(SEM_EARG, "peak_fma: iters must be in [1, 2^24]");
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = 256, blocks = sms * 8;
    void *out = dev_alloc(16);
    if (!out) return SEM_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = SEM_OK;
    for (int rep = 0; rep < 2 && rc == SEM_OK; ++rep) {  // first launch warms up
        cudaEventRecord(e0, stream());
        if (dtype == 0)
            fma_probe_kernel<double><<<blocks, threads, 0, stream()>>>(static_cast<double *>(out), iters, 0.999999, 1e-7);
        else
            fma_probe_kernel<float><<<blocks, threads, 0, stream()>>>(static_cast<float *>(out), iters, 0.999999f, 1e-7f);
        count_launches(1);
        cudaEventRecord(e1, stream());
        rc = cuda_check(cudaEventSynchronize(e1), "peak_fma");
    }
    float ms = 0.f;
    if (rc == SEM_OK) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "peak_fma: timing");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(out);
    if (rc != SEM_OK) return rc;
    *flops_per_s = 2.0 * 8.0 * double(iters) * threads * blocks / (double(ms) * 1e-3);
    return SEM_OK;
}

}  // namespace sem
