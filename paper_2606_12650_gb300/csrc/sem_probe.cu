// sem_probe.cu -- device-fact probe: sustained FMA issue rate of the FP64 and
// FP32 pipes (flops/s), for the ALU roofline of the operator kernels.  Each
// thread runs 8 independent FMA chains so that latency is hidden; the grid
// fills every SM several times over.  Also the self-test of the bounded
// device wait (wait_probe).
#include <cuda_runtime.h>

#include "sem_device.cuh"
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

// Self-test of failure detection on the GPU: one block copies 64 bytes into
// shared memory with the TMA engine and waits for them on mbarrier 0 (its
// expected byte count is exact, so the copy has landed when the wait
// returns), then waits with the bounded wait of the operator kernels on
// mbarrier 1, whose expected byte count (16) no copy ever supplies.  That
// wait gives up after ~limit_ns and sets the device status word, which the
// next sem_sync (or solve) reports as SEM_ETIMEDOUT; no copy is in flight
// when the kernel returns, and the context stays usable.
__global__ void wait_probe_kernel(const double *src, int32_t *status, uint64_t limit_ns, double *out) {
    __shared__ __align__(16) double buf[8];
    __shared__ __align__(8) uint64_t bar[2];
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&bar[0], 64);
        bulk_g2s(buf, src, 64, &bar[0]);
        mbar_arrive_expect_tx(&bar[1], 16);   // never supplied: this wait must run out
    }
    const bool copied = mbar_wait_bounded(&bar[0], 0, status);
    const bool never = mbar_wait_bounded(&bar[1], 0, status, limit_ns);
    if (threadIdx.x == 0) out[0] = copied && !never ? buf[7] : -1.0;
}

int probe_wait_timeout(uint64_t limit_ns, double *copied_value) {
    if (limit_ns < 1000 || limit_ns > 100000000ull)
        return set_error(SEM_EARG, "wait_probe: limit_ns must be in [1e3, 1e8]");
    double *buf = static_cast<double *>(dev_alloc(sizeof(double) * 16));
    if (!buf) return SEM_ENOMEM;
    double h[8] = {0, 1, 2, 3, 4, 5, 6, 7.5};
    int rc = cuda_check(cudaMemcpyAsync(buf, h, sizeof h, cudaMemcpyHostToDevice, stream()), "wait_probe: copy");
    if (rc == SEM_OK) {
        wait_probe_kernel<<<1, 32, 0, stream()>>>(buf, status_word(), limit_ns, buf + 8);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "wait_probe_kernel");
    }
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(copied_value, buf + 8, sizeof(double), cudaMemcpyDeviceToHost, stream()),
                        "wait_probe: result");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "wait_probe: sync");
    dev_free(buf);
    return rc;
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
