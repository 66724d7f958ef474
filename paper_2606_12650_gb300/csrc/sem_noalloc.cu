// sem_noalloc.cu -- sem_dot_noalloc: the weighted dot product
// sum_l c_l u_l v_l with no device allocation at all.
//
// Why it exists.  The regular "dot" kernel reduces through a partials buffer
// that libsem allocates (through cudaMalloc or the caller's allocator hook)
// when a problem is set up.  Some callers cannot let a library allocate:
// code that runs while a CUDA graph is being captured in a mode that forbids
// allocation, real-time loops that must not touch the allocator after
// start-up, and host programs whose device memory is owned by another
// framework's allocator without a hook libsem could call.  This entry point
// takes only the caller's inputs and output and keeps its scratch (per-block
// partial sums and a ticket counter) in a fixed static device array.
//
// Limits and sharing.  The array holds kMaxBlocks partials, so n may not
// exceed kMaxBlocks * kThreads * kPerThread = 16,777,216 entries; larger n is
// rejected with SEM_ERANGE.  Every GPU that loads libsem holds the 64 KB array
// until the process exits.  All calls share it and it keeps the last call's
// contents: the ticket is cleared (cudaMemsetAsync, no allocation) at the
// start of every call, and calls whose kernels overlap on the GPU (different
// streams without ordering) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "sem.h"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kMaxBlocks = 8192;
constexpr int64_t kMaxN = int64_t(kMaxBlocks) * kThreads * kPerThread;
constexpr int kTicketSlot = kMaxBlocks;  // the ticket lives in the slot after the partials
constexpr int kMaxDevices = 64;

// partials[0 .. kMaxBlocks) then one slot (viewed as uint32) for the ticket,
// padded to a 256-byte multiple
static __device__ __align__(256) double g_dot_scratch[kMaxBlocks + 32];

double *g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_lock;

__global__ void dot_noalloc_kernel(const double *__restrict__ c, const double *__restrict__ u,
                                   const double *__restrict__ v, int64_t n, double *scratch,
                                   double *out) {
    __shared__ double red[32];
    uint32_t *ticket = reinterpret_cast<uint32_t *>(scratch + kTicketSlot);
    const int64_t base = int64_t(blockIdx.x) * kThreads * kPerThread + threadIdx.x;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < kPerThread; ++q) {
        const int64_t l = base + int64_t(q) * kThreads;
        if (l < n) acc = fma(c ? c[l] * u[l] : u[l], v[l], acc);
    }
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, scratch, ticket)) {
        const double tot = finish_partials(scratch, int(gridDim.x), ticket, red);
        if (threadIdx.x == 0) *out = tot;
    }
}

// Device address of the static scratch on the current device (set up once
// per device, with that device current).
int scratch_for_current_device(double **addr) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "sem_dot_noalloc: cudaGetDevice");
    if (rc != SEM_OK) return rc;
    if (dev < 0 || dev >= kMaxDevices) return set_error(SEM_EARG, "sem_dot_noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_setup_lock);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, g_dot_scratch), "sem_dot_noalloc: cudaGetSymbolAddress");
        if (rc != SEM_OK) return rc;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *addr = g_scratch_addr[dev];
    return SEM_OK;
}

}  // namespace
}  // namespace sem

extern "C" int sem_dot_noalloc(const double *c, const double *u, const double *v, int64_t n, double *out,
                               void *stream) {
    using namespace sem;
    if (!u || !v || !out) return set_error(SEM_EARG, "sem_dot_noalloc: u, v and out must be device pointers");
    if (n < 0) return set_error(SEM_EARG, "sem_dot_noalloc: n must be >= 0");
    if (n > kMaxN)
        return set_error(SEM_ERANGE, "sem_dot_noalloc: n exceeds the static scratch limit of 16777216 entries");
    const uintptr_t mis = (reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(u) |
                           reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(out)) & 7u;
    if (mis) return set_error(SEM_EARG, "sem_dot_noalloc: arrays must be 8-byte aligned");
    double *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != SEM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    rc = cuda_check(cudaMemsetAsync(scratch + kTicketSlot, 0, sizeof(uint32_t), s), "sem_dot_noalloc: clear ticket");
    if (rc != SEM_OK) return rc;
    int64_t blocks = (n + int64_t(kThreads) * kPerThread - 1) / (int64_t(kThreads) * kPerThread);
    if (blocks < 1) blocks = 1;
    dot_noalloc_kernel<<<unsigned(blocks), kThreads, 0, s>>>(c, u, v, n, scratch, out);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "sem_dot_noalloc: launch");
}
