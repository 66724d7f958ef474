// sem_device.cuh -- device helpers: TMA bulk copies with mbarriers (bounded
// waits), deterministic block reductions, last-block tickets.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sem_internal.h"

namespace sem {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
    // make the initialised barrier visible to the async (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Wait for phase `phase` of the barrier for at most ~limit_ns.  On time-out
// the status word records it and false is returned.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, int32_t *status,
                                                  uint64_t limit_ns = 1000000000ull) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, phase)) return true;
        if (global_ns() - t0 > limit_ns) {
            if (status) atomicExch(status, (int32_t)kStatusMbarTimeout);
            return false;
        }
    }
}

// 1D bulk copy global -> shared (TMA engine), completion counted in bytes on
// the mbarrier.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Plan of a slab copy: the 16-byte-aligned middle goes through the TMA
// engine; the ragged head/tail (< 16 bytes each) through plain loads.
struct SlabPlan {
    uint32_t head_bytes;   // bytes before the first 16-byte boundary
    uint32_t mid_bytes;    // multiple of 16
    uint32_t total_bytes;
};

__device__ __forceinline__ SlabPlan slab_plan(const void *src, uint32_t bytes) {
    const uintptr_t s = reinterpret_cast<uintptr_t>(src);
    const uintptr_t t = s + bytes;
    uintptr_t s16 = (s + 15) & ~uintptr_t(15);
    uintptr_t t16 = t & ~uintptr_t(15);
    SlabPlan p;
    if (t16 <= s16) {  // no aligned middle: everything by plain loads
        p.head_bytes = bytes;
        p.mid_bytes = 0;
    } else {
        p.head_bytes = static_cast<uint32_t>(s16 - s);
        p.mid_bytes = static_cast<uint32_t>(t16 - s16);
    }
    p.total_bytes = bytes;
    return p;
}

// Returns the shared-memory address at which element 0 of a slab whose global
// source is `src` must be placed inside a 16-byte-aligned buffer `buf` so that
// the aligned middle lands on a 16-byte boundary.
template <typename T>
__device__ __forceinline__ T *slab_dst(void *buf, const T *src) {
    const uintptr_t mis = reinterpret_cast<uintptr_t>(src) & 15u;
    return reinterpret_cast<T *>(static_cast<unsigned char *>(buf) + mis);
}

// Issue the TMA part of a slab copy (one thread).
template <typename T>
__device__ __forceinline__ void slab_issue(T *dst, const T *src, const SlabPlan &p,
                                           uint64_t *bar) {
    if (p.mid_bytes) {
        const unsigned char *s = reinterpret_cast<const unsigned char *>(src) + p.head_bytes;
        unsigned char *d = reinterpret_cast<unsigned char *>(dst) + p.head_bytes;
        bulk_g2s(d, s, p.mid_bytes, bar);
    }
}

// Have the TMA engine bring the 16-byte-aligned middle of [src, src + bytes)
// into L2: no destination and no completion to wait for, and no byte outside
// the range is touched.  One thread.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    const SlabPlan p = slab_plan(src, bytes);
    if (p.mid_bytes)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                         reinterpret_cast<const unsigned char *>(src) + p.head_bytes),
                     "r"(p.mid_bytes)
                     : "memory");
}

// Plain-load part of a slab copy (ragged head and tail), element-wise,
// spread over threads [t0, t0 + nthreads).
template <typename T>
__device__ __forceinline__ void slab_edges(T *dst, const T *src, const SlabPlan &p, int t,
                                           int nthreads) {
    const uint32_t n_head = p.head_bytes / sizeof(T);
    const uint32_t n_tot = p.total_bytes / sizeof(T);
    const uint32_t tail0 = (p.head_bytes + p.mid_bytes) / sizeof(T);
    for (uint32_t q = t; q < n_head; q += nthreads) dst[q] = src[q];
    for (uint32_t q = tail0 + t; q < n_tot; q += nthreads) dst[q] = src[q];
}

// Deterministic block sum (fixed shuffle tree, then fixed cross-warp tree).
// blockDim.x must be a multiple of 32.  The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sbuf /* >= 32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sbuf[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? sbuf[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// Deterministic block sum with few FP64 operations: every thread's value
// goes to shared memory, one warp adds them in a fixed order (strided per
// lane, then a shuffle tree).  scratch: >= blockDim.x doubles of shared
// memory that no thread still uses (the call begins with a barrier).  For
// kernels whose other arithmetic is FP32, where the per-warp shuffle tree of
// block_sum would keep the FP64 pipe (1/64 of the FP32 rate on GB300) busy
// at every block's end.  Result in thread 0.
__device__ __forceinline__ double block_sum_wide(double v, double *scratch) {
    __syncthreads();
    scratch[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (int q = threadIdx.x; q < blockDim.x; q += 32) s += scratch[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// Publish this block's partial and find out whether it is the last block to
// do so.  Thread 0 writes partials[blockIdx.x]; all threads get the answer.
__device__ __forceinline__ bool publish_partial(double v0, double *partials, uint32_t *ticket) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v0;
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return s_last != 0;
}

// In the last block: sum partials[0..n) in a fixed order (strided per thread,
// then block_sum).  Resets the ticket for the next launch.  Result in thread 0.
__device__ __forceinline__ double finish_partials(const double *partials, int n, uint32_t *ticket,
                                                  double *sbuf) {
    __threadfence();
    double acc = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) acc += __ldcg(partials + q);
    acc = block_sum(acc, sbuf);
    if (threadIdx.x == 0) *ticket = 0u;
    return acc;
}

// Two-level grid sum for launches of many blocks.  Each block publishes into
// its group of kSumGroup consecutive blocks; the group's last block to arrive
// sums the group's partials in order (one warp, fixed shuffle tree), stores
// the group sum, resets the group ticket and takes a ticket of the grid; the
// last group returns true in all threads of its block, and finish_grouped
// then sums the group sums in order.  The FP64 additions of the grid sum are
// spread over the groups' last blocks instead of all falling on one block at
// the end of the launch (on GB300 FP64 runs at 1/64 of the FP32 rate).
__device__ __forceinline__ bool publish_grouped(double v0, double *partials, uint32_t *ticket) {
    __shared__ int s_last;
    const int64_t cap = partials_capacity(partials);
    uint32_t *gt = group_tickets(partials, cap);
    const int b = int(blockIdx.x), g = b / kSumGroup, g0 = g * kSumGroup;
    const int gn = min(kSumGroup, int(gridDim.x) - g0);
    if (threadIdx.x == 0) {
        partials[b] = v0;
        __threadfence();
        s_last = atomicAdd(gt + g, 1u) == uint32_t(gn - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __syncthreads();  // every thread has read s_last before thread 0 rewrites it
    if (threadIdx.x < 32) {
        __threadfence();
        double s = int(threadIdx.x) < gn ? __ldcg(partials + g0 + threadIdx.x) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) {
            partials[cap + g] = s;
            gt[g] = 0u;
            __threadfence();
            const uint32_t ng = (gridDim.x + kSumGroup - 1) / kSumGroup;
            s_last = atomicAdd(ticket, 1u) == ng - 1;
        }
    }
    __syncthreads();
    return s_last != 0;
}

// Zero the group tickets (grid-stride): at the start of every solve, so that
// a launch that gave up half-way (a timed-out copy) leaves no stale count.
__device__ __forceinline__ void reset_group_tickets(double *partials) {
    const int64_t cap = partials_capacity(partials);
    uint32_t *gt = group_tickets(partials, cap);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < cap / kSumGroup;
         i += int64_t(gridDim.x) * blockDim.x)
        gt[i] = 0u;
}

// In the block for which publish_grouped returned true: the sum of the group
// sums in a fixed order (one warp), the grid ticket reset.  Result in thread 0.
__device__ __forceinline__ double finish_grouped(const double *partials, uint32_t *ticket) {
    double s = 0.0;
    if (threadIdx.x < 32) {
        __threadfence();
        const int ng = int((gridDim.x + kSumGroup - 1) / kSumGroup);
        const int64_t cap = partials_capacity(partials);
        for (int q = threadIdx.x; q < ng; q += 32) s += __ldcg(partials + cap + q);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *ticket = 0u;
    }
    return s;
}

// Block sum of FP32 values in FP32: fixed shuffle tree per warp, then the
// warp sums in order by warp 0.  scratch: >= 32 floats of shared memory that
// the block may still be reading (the first barrier protects it).  Result in
// thread 0.
__device__ __forceinline__ float block_sum_f32(float v, float *scratch) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    float s = 0.f;
    if (wid == 0) {
        s = lane < nw ? scratch[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// Two-value variants (PCG: <r, z> and <r, r>): slots partials[2b], [2b+1].
__device__ __forceinline__ bool publish_partial2(double v0, double v1, double *partials, uint32_t *ticket) {
    __shared__ int s_last2;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = v0;
        partials[2 * blockIdx.x + 1] = v1;
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        s_last2 = (t == gridDim.x - 1);
    }
    __syncthreads();
    return s_last2 != 0;
}

__device__ __forceinline__ void finish_partials2(const double *partials, int n, uint32_t *ticket, double *sbuf,
                                                 double *t0, double *t1) {
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        a += __ldcg(partials + 2 * q);
        b += __ldcg(partials + 2 * q + 1);
    }
    a = block_sum(a, sbuf);
    b = block_sum(b, sbuf);
    if (threadIdx.x == 0) {
        *ticket = 0u;
        *t0 = a;
        *t1 = b;
    }
}

// Closing step of a PCG iteration (thread 0 of the last block): rho_new =
// <r, M^-1 r> drives beta, rr = <r, r> the stop test sqrt(rr / bb) <= tol.
__device__ __forceinline__ void pcg_close_iteration(CgState *st, double rho_new, double rr) {
    const int it = st->iter + 1;
    st->iter = it;
    st->rr = rr;
    if (st->hist) st->hist[it] = sqrt(rr);
    const double rho = st->rho;
    st->beta = rho_new / rho;
    st->rho = rho_new;
    const bool conv = st->tol > 0.0 && sqrt(rr / st->bb) <= st->tol;
    if (conv || it >= st->maxit) st->done = 1;
}

// Closing step of a CG iteration, run by thread 0 of the last block once
// rho_new = <r_{k+1}, r_{k+1}> is known: iteration count, optional history,
// beta = rho_new / rho, and the stop flag (relative residual or maxit).
__device__ __forceinline__ void cg_close_iteration(CgState *st, double rho_new) {
    const int it = st->iter + 1;
    st->iter = it;
    if (st->hist) st->hist[it] = sqrt(rho_new);
    const double rho = st->rho;
    st->beta = rho_new / rho;
    st->rho = rho_new;
    const bool conv = st->tol > 0.0 && sqrt(rho_new / st->rho0) <= st->tol;
    if (conv || it >= st->maxit) st->done = 1;
}

}  // namespace sem
