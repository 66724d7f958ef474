// sem_batch.cu -- many independent Poisson problems of different sizes and
// orders solved together: each CG phase is ONE persistent launch over all
// problems, replayed from a CUDA graph.
//
// Work lists.  Every problem is cut into operator items (groups of up to EPB(N)
// elements, EPB(N) = 256 / (N+1)^2) and vector items (row-aligned runs of
// ~4096 local nodes).  A persistent kernel's CTAs take items from a global
// counter (dynamic load balance across problems of very different cost); a
// device-side switch on N dispatches to the body compiled for that order.
//
// Per-problem reductions.  Each item writes one partial (fixed-order block
// tree) to its own slot; the problem's last item to finish (per-problem
// ticket) sums the problem's slots in item order.  The items of a problem and
// the trees inside them do not depend on which other problems share the
// batch, so a problem's iterates are bit-identical alone or in any mix.
//
// States.  Each problem has its own CG state (and an inner one for mixed
// precision); finished problems turn their items into no-ops, and a device
// counter of finished problems is polled once per graph replay.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "sem_ax_kernel.cuh"
#include "sem_box.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kBatchThreads = 256;
constexpr int kVecItemNodes = 4096;

struct BatchProb {
    int nq, nx, ny, nz;
    int64_t E, nL;
    int64_t off;                    // offset in the concatenated b / x arrays
    const double *G;
    const __nv_bfloat16 *G16;
    const float *G32;
    const double *c;
    double *x, *r, *p, *w;          // FP64 CG vectors / refinement x, r
    float *d32, *r32, *p32, *w32;   // inner (FP32) CG vectors
    CgState *st, *st_in;
    int ax_first, ax_count;         // operator items
    int vec_first, vec_count;       // vector items
    int32_t outer_done;             // mixed: true residual reached tol
    int32_t inner_total;            // mixed: inner iterations so far
    double bb;                      // <b, b>_c
    double res;                     // mixed: current true relative residual
};

struct BatchItem {
    int prob, nq;
    int64_t first;  // first element (operator) or first local node (vector)
    int count;      // elements or nodes
    int pad;
};

struct BatchQueue {
    unsigned next, exited, pad0, pad1;
};

enum BatchQ : int { kQAx = 0, kQVec = 1, kNumQ = 2 };

struct BatchCtl {
    BatchQueue q[kNumQ];
    unsigned n_done;                // problems whose (inner) CG finished
    unsigned n_outer_done;          // mixed: problems whose true residual reached tol
    unsigned pad[2];
};

struct Batch {
    std::vector<Problem *> probs;
    std::vector<int64_t> offs;
    int64_t nL_total = 0;
    int n_ax = 0, n_vec = 0;
    BatchProb *d_probs = nullptr;
    BatchItem *d_ax = nullptr, *d_vec = nullptr;
    double *part = nullptr;         // one slot per item
    uint32_t *tickets = nullptr;    // per problem: [ax, vec]
    BatchCtl *ctl = nullptr;
    BatchCtl *ctl_host = nullptr;
    int grid_ax64 = 0, grid_ax32 = 0, grid_vec = 0;
    cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};   // FP64 CG, inner bf16, inner f32
    int graph_iters = 0;
    cudaStream_t graph_stream = nullptr;
};

// ------------------------------------------------------------------ shapes
template <int NQ>
struct BEpb {
    static constexpr int value = kBatchThreads / (NQ * NQ);
};

template <typename T>
constexpr size_t batch_ax_smem() {
    size_t m = 0;
#define SEM_BS(Q) m = std::max(m, AxShape<Q, BEpb<Q>::value, T>::SMEM);
    SEM_BS(2) SEM_BS(3) SEM_BS(4) SEM_BS(5) SEM_BS(6) SEM_BS(7) SEM_BS(8) SEM_BS(9) SEM_BS(10)
#undef SEM_BS
    return m;
}

// Derivative matrices of every order in constant memory: D depends only on
// N, so inside the switch case for order N every index is a compile-time
// constant and the products read constant-bank operands directly.
__constant__ double c_D64[kMaxQ - 1][kMaxQ * kMaxQ];
__constant__ float c_D32[kMaxQ - 1][kMaxQ * kMaxQ];

template <int NQ, typename T>
struct ConstD;
template <int NQ>
struct ConstD<NQ, double> {
    __device__ __forceinline__ double operator[](int q) const { return c_D64[NQ - 2][q]; }
};
template <int NQ>
struct ConstD<NQ, float> {
    __device__ __forceinline__ float operator[](int q) const { return c_D32[NQ - 2][q]; }
};

template <typename GT>
__device__ __forceinline__ const GT *prob_G(const BatchProb &P);
template <> __device__ __forceinline__ const double *prob_G<double>(const BatchProb &P) { return P.G; }
template <> __device__ __forceinline__ const __nv_bfloat16 *prob_G<__nv_bfloat16>(const BatchProb &P) { return P.G16; }
template <> __device__ __forceinline__ const float *prob_G<float>(const BatchProb &P) { return P.G32; }

// Take the next item from a queue (thread 0), broadcast to the block.
__device__ __forceinline__ int next_item(BatchQueue *q, int *s_item) {
    if (threadIdx.x == 0) *s_item = int(atomicAdd(&q->next, 1u));
    __syncthreads();
    const int it = *s_item;
    __syncthreads();
    return it;
}

// The last CTA to leave resets the queue for the next launch.
__device__ __forceinline__ void leave_queue(BatchQueue *q) {
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&q->exited, 1u) == gridDim.x - 1) {
            q->next = 0;
            q->exited = 0;
            __threadfence();
        }
    }
}

// Publish an item's partial; if it is the problem's last item, return true
// and the problem's total (items summed in order) in *total (thread 0).
__device__ __forceinline__ bool item_partial(double v0, double *part, int it, uint32_t *ticket, int first,
                                             int count, double *sbuf, double *total) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        part[it] = v0;
        __threadfence();
        s_last = (atomicAdd(ticket, 1u) == unsigned(count) - 1u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int q = threadIdx.x; q < count; q += blockDim.x) acc += __ldcg(part + first + q);
    acc = block_sum(acc, sbuf);
    if (threadIdx.x == 0) {
        *ticket = 0u;
        *total = acc;
    }
    return true;
}

// ------------------------------------------------------------------ operator
// One item of order NQ.  Kept out of line so that each order's body gets its
// own register allocation (inlined into one switch, the nine bodies share and
// exhaust the register file).
template <int NQ, typename T, typename GT, bool CG>
__device__ __noinline__ bool batch_ax_item(const T *xin, T *yout, T *pv, const GT *G, T beta, int64_t first,
                                           int count, T *regA, uint64_t *bar, uint32_t phase, int32_t *status,
                                           T *pt) {
    return ax_group<NQ, BEpb<NQ>::value, T, GT, CG>(xin, yout, pv, G, ConstD<NQ, T>{}, beta, first, count, regA,
                                                   bar, phase, status, pt);
}

// mode: 0 = FP64 CG (p = r + beta p, w = A p), 1 = FP64 plain (w = A x),
//       2 = FP32 inner CG on the FP32 vectors
template <typename T, typename GT, int MODE>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_ax_kernel(BatchProb *probs, const BatchItem *items,
                                                                 int nitems, double *part, uint32_t *tickets,
                                                                 BatchCtl *ctl, int32_t *status) {
    constexpr bool CG = MODE != 1;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_item;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *regA = reinterpret_cast<T *>(smem + 16);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    BatchQueue *q = &ctl->q[kQAx];
    while (true) {
        const int it = next_item(q, &s_item);
        if (it >= nitems) break;
        const BatchItem item = items[it];
        BatchProb &P = probs[item.prob];
        CgState *st = MODE == 2 ? P.st_in : P.st;
        if (CG && st->done) continue;
        if (MODE == 1 && P.outer_done) continue;   // refinement: converged problems need no residual
        const T beta = CG ? T(st->beta) : T(0);
        const T *xin;
        T *yout, *pv;
        if (MODE == 0) { xin = reinterpret_cast<const T *>(P.r); yout = reinterpret_cast<T *>(P.w); pv = reinterpret_cast<T *>(P.p); }
        else if (MODE == 1) { xin = reinterpret_cast<const T *>(P.x); yout = reinterpret_cast<T *>(P.w); pv = nullptr; }
        else { xin = reinterpret_cast<const T *>(P.r32); yout = reinterpret_cast<T *>(P.w32); pv = reinterpret_cast<T *>(P.p32); }
        const GT *G = prob_G<GT>(P);
        T pt = T(0);
        bool ok = true, used = true;
        switch (item.nq) {
#define SEM_BAX(Q)                                                                                     \
    case Q:                                                                                            \
        ok = batch_ax_item<Q, T, GT, CG>(xin, yout, pv, G, beta, item.first, item.count, regA, bar,     \
                                         phase, status, &pt);                                          \
        break;
            SEM_BAX(2) SEM_BAX(3) SEM_BAX(4) SEM_BAX(5) SEM_BAX(6) SEM_BAX(7) SEM_BAX(8) SEM_BAX(9) SEM_BAX(10)
#undef SEM_BAX
            default: used = false; break;
        }
        if (used) phase ^= 1u;
        if (!ok) return;  // timed out: the status word reports it; the solve is abandoned
        if (CG) {
            const double bs = block_sum(double(pt), red);
            double pap;
            if (item_partial(bs, part, it, &tickets[2 * item.prob], P.ax_first, P.ax_count, red, &pap) &&
                threadIdx.x == 0) {
                st->pap = pap;
                st->alpha = st->rho / pap;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    leave_queue(q);
}

// ------------------------------------------------------------------ vector phases
enum VecMode : int {
    kVecUpdate64 = 0,   // FP64 CG update (gs of w, x/r update, <r,r>, close)
    kVecUpdate32 = 1,   // FP32 inner CG update
    kVecInit64 = 2,     // x = 0, p = 0, r = b, <b,b> -> CG state
    kVecInner = 3,      // r32 = r, d32 = p32 = 0, <r32,r32> -> inner state
    kVecCorrect = 4,    // x += d32
    kVecResidual = 5,   // r = b - mask(QQ^T w), <r,r> -> outer test
    kVecCopyOut = 6,    // xout = x
};

struct VecArgs {
    const double *b_all;
    double *x_all;
    double tol;         // outer tolerance (residual test), or CG tolerance (init)
    double inner_tol;   // minimum inner reduction (mixed)
    int maxit;
};

// r = b - mask(QQ^T w) at one node (box-structured copies, ascending order),
// returns the node's <r, r> contribution (first copy only).
template <int NQ>
__device__ __forceinline__ double residual_node(double *r, const double *b, const double *w, int l, int nx, int ny,
                                                int nz) {
    const BoxNode bn = box_node<NQ>(l, nx, ny, nz);
    if (bn.masked) {
        r[l] = 0.0;
        return 0.0;
    }
    const int z0 = bn.sz < 0 ? bn.oz : 0, z1 = bn.sz > 0 ? bn.oz : 0;
    const int y0 = bn.sy < 0 ? bn.oy : 0, y1 = bn.sy > 0 ? bn.oy : 0;
    const int x0 = bn.sx < 0 ? bn.ox : 0, x1 = bn.sx > 0 ? bn.ox : 0;
    double s = 0.0;
    bool first = true;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int cz = c >> 2, cy = (c >> 1) & 1, cx = c & 1;
        if (!((cz == 0 || bn.sz) && (cy == 0 || bn.sy) && (cx == 0 || bn.sx))) continue;
        const double v = __ldg(w + l + (cz ? z1 : z0) + (cy ? y1 : y0) + (cx ? x1 : x0));
        s = first ? v : s + v;
        first = false;
    }
    const double rv = b[l] - s;
    r[l] = rv;
    return bn.owner ? rv * rv : 0.0;
}

template <int NQ, int MODE>
__device__ __noinline__ double vec_item_body(BatchProb &P, CgState *st, const VecArgs &A, int64_t first,
                                                int count) {
    double acc = 0.0;
    const int tid = threadIdx.x;
    if (MODE == kVecUpdate64 || MODE == kVecUpdate32) {
        using T = typename std::conditional<MODE == kVecUpdate64, double, float>::type;
        constexpr int V = UpdVec<NQ, T>::value;
        T *x = MODE == kVecUpdate64 ? reinterpret_cast<T *>(P.x) : reinterpret_cast<T *>(P.d32);
        T *r = MODE == kVecUpdate64 ? reinterpret_cast<T *>(P.r) : reinterpret_cast<T *>(P.r32);
        const T *p = MODE == kVecUpdate64 ? reinterpret_cast<const T *>(P.p) : reinterpret_cast<const T *>(P.p32);
        const T *w = MODE == kVecUpdate64 ? reinterpret_cast<const T *>(P.w) : reinterpret_cast<const T *>(P.w32);
        const T alpha = T(st->alpha);
        T a = T(0);
        for (int v = tid; v < count / V; v += blockDim.x)
            a += update_vec<NQ, V, T, T>(x, r, p, w, int(first) + v * V, P.nx, P.ny, P.nz, alpha);
        acc = double(a);
    } else if (MODE == kVecInit64) {
        const double *b = A.b_all + P.off;
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            const double bl = b[l];
            P.x[l] = 0.0;
            P.p[l] = 0.0;
            P.r[l] = bl;
            acc = fma(P.c[l] * bl, bl, acc);
        }
    } else if (MODE == kVecInner) {
        if (P.outer_done) return 0.0;   // converged: the inner state is closed in the handler
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            const float f = __double2float_rn(P.r[l]);
            P.r32[l] = f;
            P.d32[l] = 0.f;
            P.p32[l] = 0.f;
            acc += P.c[l] * double(f) * double(f);
        }
    } else if (MODE == kVecCorrect) {
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            P.x[l] += double(P.d32[l]);
        }
    } else if (MODE == kVecResidual) {
        const double *b = A.b_all + P.off;
        for (int v = tid; v < count; v += blockDim.x)
            acc += residual_node<NQ>(P.r, b, P.w, int(first) + v, P.nx, P.ny, P.nz);
    } else if (MODE == kVecCopyOut) {
        double *xo = A.x_all + P.off;
        for (int v = tid; v < count; v += blockDim.x) xo[first + v] = P.x[first + v];
    }
    return acc;
}

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads, 3) batch_vec_kernel(BatchProb *probs, const BatchItem *items,
                                                                  int nitems, double *part, uint32_t *tickets,
                                                                  BatchCtl *ctl, VecArgs A) {
    __shared__ double red[32];
    __shared__ int s_item;
    constexpr bool REDUCES = MODE != kVecCorrect && MODE != kVecCopyOut;
    BatchQueue *q = &ctl->q[kQVec];
    while (true) {
        const int it = next_item(q, &s_item);
        if (it >= nitems) break;
        const BatchItem item = items[it];
        BatchProb &P = probs[item.prob];
        CgState *st = (MODE == kVecUpdate32 || MODE == kVecInner) ? P.st_in : P.st;
        // skip finished problems (their items are no-ops)
        if (MODE == kVecUpdate64 || MODE == kVecUpdate32) {
            if (st->done) continue;
        } else if (MODE == kVecCorrect || MODE == kVecResidual) {
            if (P.outer_done) continue;
        }
        double acc = 0.0;
        switch (item.nq) {
#define SEM_BV(Q)                                                          \
    case Q:                                                                \
        acc = vec_item_body<Q, MODE>(P, st, A, item.first, item.count);    \
        break;
            SEM_BV(2) SEM_BV(3) SEM_BV(4) SEM_BV(5) SEM_BV(6) SEM_BV(7) SEM_BV(8) SEM_BV(9) SEM_BV(10)
#undef SEM_BV
            default: break;
        }
        if (!REDUCES) continue;
        const double bs = block_sum(acc, red);
        double tot;
        if (item_partial(bs, part, it, &tickets[2 * item.prob + 1], P.vec_first, P.vec_count, red, &tot) &&
            threadIdx.x == 0) {
            if (MODE == kVecUpdate64 || MODE == kVecUpdate32) {
                cg_close_iteration(st, tot);
                if (st->done) atomicAdd(&ctl->n_done, 1u);
            } else if (MODE == kVecInit64) {
                st->rho = tot;
                st->rho0 = tot;
                st->alpha = st->beta = st->pap = 0.0;
                st->tol = A.tol;
                st->hist = nullptr;
                st->iter = 0;
                st->maxit = A.maxit;
                st->done = (tot == 0.0 || A.maxit <= 0) ? 1 : 0;
                P.bb = tot;
                P.res = tot > 0.0 ? 1.0 : 0.0;
                P.outer_done = (tot == 0.0) ? 1 : 0;
                P.inner_total = 0;
                if (st->done) atomicAdd(&ctl->n_done, 1u);
                if (P.outer_done) atomicAdd(&ctl->n_outer_done, 1u);
            } else if (MODE == kVecInner) {
                if (P.outer_done) {
                    st->done = 1;   // not counted: only problems still refining are waited for
                    st->iter = 0;
                } else {
                    const double eta = fmin(0.5, fmax(A.inner_tol, 0.5 * A.tol / P.res));
                    st->rho = tot;
                    st->rho0 = tot;
                    st->alpha = st->beta = st->pap = 0.0;
                    st->tol = eta;
                    st->hist = nullptr;
                    st->iter = 0;
                    st->maxit = A.maxit;
                    st->done = (tot == 0.0) ? 1 : 0;
                    if (st->done) atomicAdd(&ctl->n_done, 1u);
                }
            } else if (MODE == kVecResidual) {
                P.inner_total += P.st_in->iter;
                P.res = P.bb > 0.0 ? sqrt(tot / P.bb) : 0.0;
                P.st->rho = tot;
                if (P.res <= A.tol) {
                    P.outer_done = 1;
                    atomicAdd(&ctl->n_outer_done, 1u);
                }
            }
        }
    }
    leave_queue(q);
}

// ------------------------------------------------------------------ host side
static int batch_grid(const void *kern, size_t smem, int *out) {
    int per_sm = 0;
    const int rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem),
                              "batch: occupancy");
    if (rc != SEM_OK) return rc;
    if (per_sm < 1) return set_error(SEM_ECUDA, "batch: kernel does not fit on an SM");
    *out = per_sm * sm_count();
    return SEM_OK;
}

template <typename T, typename GT, int MODE>
static int launch_bax(Batch *B, int grid) {
    constexpr size_t sm = batch_ax_smem<T>();
    batch_ax_kernel<T, GT, MODE><<<unsigned(grid), kBatchThreads, sm, stream()>>>(
        B->d_probs, B->d_ax, B->n_ax, B->part, B->tickets, B->ctl, status_word());
    count_launches(1);
    return cuda_check(cudaGetLastError(), "batch_ax_kernel");
}

template <int MODE>
static int launch_bvec(Batch *B, const VecArgs &A) {
    batch_vec_kernel<MODE><<<unsigned(B->grid_vec), kBatchThreads, 0, stream()>>>(B->d_probs, B->d_vec, B->n_vec,
                                                                                B->part, B->tickets, B->ctl, A);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "batch_vec_kernel");
}

static int batch_attrs(Batch *B) {
    static bool done = false;
    if (!done) {
        static double h64[kMaxQ - 1][kMaxQ * kMaxQ];
        static float h32[kMaxQ - 1][kMaxQ * kMaxQ];
        for (int N = 1; N <= kMaxQ - 1; ++N) {
            double xi[kMaxQ], w[kMaxQ];
            gll_rule_and_derivative(N, xi, w, h64[N - 1]);
            for (int q = 0; q < (N + 1) * (N + 1); ++q) h32[N - 1][q] = float(h64[N - 1][q]);
        }
        int rc0 = cuda_check(cudaMemcpyToSymbol(c_D64, h64, sizeof h64), "batch: D table");
        if (rc0 == SEM_OK) rc0 = cuda_check(cudaMemcpyToSymbol(c_D32, h32, sizeof h32), "batch: D table");
        if (rc0 != SEM_OK) return rc0;
        const int a = int(batch_ax_smem<double>()), f = int(batch_ax_smem<float>());
        int rc = cuda_check(cudaFuncSetAttribute(batch_ax_kernel<double, double, 0>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, a), "batch attr");
        if (rc == SEM_OK)
            rc = cuda_check(cudaFuncSetAttribute(batch_ax_kernel<double, double, 1>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, a), "batch attr");
        if (rc == SEM_OK)
            rc = cuda_check(cudaFuncSetAttribute(batch_ax_kernel<float, __nv_bfloat16, 2>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, f), "batch attr");
        if (rc == SEM_OK)
            rc = cuda_check(cudaFuncSetAttribute(batch_ax_kernel<float, float, 2>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, f), "batch attr");
        if (rc != SEM_OK) return rc;
        done = true;
    }
    int rc = batch_grid(reinterpret_cast<const void *>(batch_ax_kernel<double, double, 0>), batch_ax_smem<double>(),
                        &B->grid_ax64);
    if (rc == SEM_OK)
        rc = batch_grid(reinterpret_cast<const void *>(batch_ax_kernel<float, __nv_bfloat16, 2>),
                        batch_ax_smem<float>(), &B->grid_ax32);
    if (rc == SEM_OK)
        rc = batch_grid(reinterpret_cast<const void *>(batch_vec_kernel<kVecUpdate64>), 0, &B->grid_vec);
    return rc;
}

int batch_create(Problem **probs, int n, Batch **out) {
    *out = nullptr;
    if (n < 1) return set_error(SEM_EARG, "batch: needs at least one problem");
    Batch *B = new Batch();
    B->probs.assign(probs, probs + n);
    std::vector<BatchProb> hp(n);
    std::vector<BatchItem> ax, vec;
    int rc = SEM_OK;
    int64_t off = 0;
    for (int k = 0; k < n && rc == SEM_OK; ++k) {
        Problem *P = probs[k];
        rc = mixed_prepare(P, kGBF16);
        if (rc == SEM_OK) rc = mixed_prepare(P, kGF32);
        if (rc != SEM_OK) break;
        BatchProb &q = hp[k];
        memset(&q, 0, sizeof q);
        q.nq = P->nq; q.nx = P->nx; q.ny = P->ny; q.nz = P->nz;
        q.E = P->E; q.nL = P->nL; q.off = off;
        q.G = P->G; q.G16 = static_cast<const __nv_bfloat16 *>(P->G16); q.G32 = static_cast<const float *>(P->G32);
        q.c = P->c;
        q.x = P->x; q.r = P->r; q.p = P->p; q.w = P->w;
        q.d32 = P->d32; q.r32 = P->r32; q.p32 = P->p32; q.w32 = P->w32;
        q.st = P->st; q.st_in = P->st_in;
        const int epb = kBatchThreads / (P->nq * P->nq);
        q.ax_first = int(ax.size());
        for (int64_t e = 0; e < P->E; e += epb)
            ax.push_back(BatchItem{k, P->nq, e, int(std::min<int64_t>(epb, P->E - e)), 0});
        q.ax_count = int(ax.size()) - q.ax_first;
        // vector items: row-aligned runs of about kVecItemNodes nodes
        const int64_t chunk = std::max<int64_t>(P->nq, (kVecItemNodes / P->nq) * P->nq);
        q.vec_first = int(vec.size());
        for (int64_t l = 0; l < P->nL; l += chunk)
            vec.push_back(BatchItem{k, P->nq, l, int(std::min<int64_t>(chunk, P->nL - l)), 0});
        q.vec_count = int(vec.size()) - q.vec_first;
        B->offs.push_back(off);
        off += P->nL;
    }
    B->nL_total = off;
    B->n_ax = int(ax.size());
    B->n_vec = int(vec.size());
    if (rc == SEM_OK) {
        B->d_probs = static_cast<BatchProb *>(dev_alloc(sizeof(BatchProb) * n));
        B->d_ax = static_cast<BatchItem *>(dev_alloc(sizeof(BatchItem) * ax.size()));
        B->d_vec = static_cast<BatchItem *>(dev_alloc(sizeof(BatchItem) * vec.size()));
        B->part = static_cast<double *>(dev_alloc(sizeof(double) * std::max(ax.size(), vec.size())));
        B->tickets = static_cast<uint32_t *>(dev_alloc(sizeof(uint32_t) * 2 * n));
        B->ctl = static_cast<BatchCtl *>(dev_alloc(sizeof(BatchCtl)));
        if (!B->d_probs || !B->d_ax || !B->d_vec || !B->part || !B->tickets || !B->ctl) rc = SEM_ENOMEM;
    }
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B->d_probs, hp.data(), sizeof(BatchProb) * n, cudaMemcpyHostToDevice, stream()),
                        "batch: descriptors");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B->d_ax, ax.data(), sizeof(BatchItem) * ax.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B->d_vec, vec.data(), sizeof(BatchItem) * vec.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(B->tickets, 0, sizeof(uint32_t) * 2 * n, stream()), "batch");
    if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(B->ctl, 0, sizeof(BatchCtl), stream()), "batch");
    if (rc == SEM_OK) rc = cuda_check(cudaMallocHost(&B->ctl_host, sizeof(BatchCtl)), "batch: pinned");
    if (rc == SEM_OK) rc = batch_attrs(B);
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc != SEM_OK) {
        batch_destroy(B);
        return rc;
    }
    *out = B;
    return SEM_OK;
}

void batch_destroy(Batch *B) {
    if (!B) return;
    for (auto &g : B->graph)
        if (g) cudaGraphExecDestroy(g);
    void *ptrs[] = {B->d_probs, B->d_ax, B->d_vec, B->part, B->tickets, B->ctl};
    for (void *q : ptrs)
        if (q) dev_free(q);
    if (B->ctl_host) cudaFreeHost(B->ctl_host);
    delete B;
}

int64_t batch_total_nodes(const Batch *B) { return B->nL_total; }
int batch_size(const Batch *B) { return int(B->probs.size()); }

static int read_ctl(Batch *B) {
    int rc = cuda_check(cudaMemcpyAsync(B->ctl_host, B->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, stream()),
                        "batch: control read");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc == SEM_OK) rc = poll_status();
    return rc;
}

static int reset_done(Batch *B) {
    return cuda_check(cudaMemsetAsync(&B->ctl->n_done, 0, sizeof(unsigned), stream()), "batch: reset");
}

// K iterations of (operator, update) for one precision, captured once.
static int capture(Batch *B, int which) {
    if (B->graph[which] && B->graph_stream == stream()) return SEM_OK;
    if (B->graph[which]) {
        cudaGraphExecDestroy(B->graph[which]);
        B->graph[which] = nullptr;
    }
    const int K = B->nL_total < (int64_t(1) << 22) ? 64 : 16;
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(stream(), cudaStreamCaptureModeThreadLocal), "batch: capture");
    if (rc != SEM_OK) return rc;
    const VecArgs none{};
    for (int k = 0; k < K && rc == SEM_OK; ++k) {
        if (which == 0) {
            rc = launch_bax<double, double, 0>(B, B->grid_ax64);
            if (rc == SEM_OK) rc = launch_bvec<kVecUpdate64>(B, none);
        } else {
            rc = which == 1 ? launch_bax<float, __nv_bfloat16, 2>(B, B->grid_ax32)
                            : launch_bax<float, float, 2>(B, B->grid_ax32);
            if (rc == SEM_OK) rc = launch_bvec<kVecUpdate32>(B, none);
        }
    }
    count_launches(-2 * int64_t(K));
    const int rc_end = cuda_check(cudaStreamEndCapture(stream(), &g), "batch: end capture");
    if (rc == SEM_OK) rc = rc_end;
    if (rc == SEM_OK) rc = cuda_check(cudaGraphInstantiate(&B->graph[which], g, 0), "batch: instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc == SEM_OK) {
        B->graph_iters = K;
        B->graph_stream = stream();
    }
    return rc;
}

// Replay the captured iterations until every problem's (inner) CG has
// stopped or maxit iterations have run.
static int run_until_done(Batch *B, int which, int maxit, unsigned target) {
    const int64_t max_replays = (int64_t(maxit) + B->graph_iters - 1) / B->graph_iters;
    for (int64_t rep = 0; rep < max_replays; ++rep) {
        int rc = read_ctl(B);
        if (rc != SEM_OK) return rc;
        if (B->ctl_host->n_done >= target) return SEM_OK;
        rc = cuda_check(cudaGraphLaunch(B->graph[which], stream()), "batch: graph launch");
        if (rc != SEM_OK) return rc;
        count_launches(2 * int64_t(B->graph_iters));
    }
    return read_ctl(B);
}

int batch_solve(Batch *B, const double *b_all, double *x_all, double tol, int maxit, int mode, double inner_tol,
                int max_outer, int64_t *iters, double *res) {
    if (mode < 0 || mode > 2) return set_error(SEM_EARG, "batch_solve: mode must be 0 (fp64), 1 (bf16), 2 (fp32)");
    if (maxit < 1) return set_error(SEM_EARG, "batch_solve: maxit must be >= 1");
    const int n = batch_size(B);
    VecArgs A{b_all, x_all, tol, inner_tol, maxit};
    int rc = cuda_check(cudaMemsetAsync(B->ctl, 0, sizeof(BatchCtl), stream()), "batch: reset");
    if (rc == SEM_OK) rc = launch_bvec<kVecInit64>(B, A);
    if (rc != SEM_OK) return rc;
    if (mode == 0) {
        rc = capture(B, 0);
        if (rc == SEM_OK) rc = run_until_done(B, 0, maxit, unsigned(n));
    } else {
        rc = capture(B, mode);
        for (int outer = 0; outer < max_outer && rc == SEM_OK; ++outer) {
            rc = read_ctl(B);
            if (rc != SEM_OK || B->ctl_host->n_outer_done >= unsigned(n)) break;
            // inner solves still to finish: the problems not yet converged
            const unsigned need = unsigned(n) - B->ctl_host->n_outer_done;
            rc = reset_done(B);
            if (rc == SEM_OK) rc = launch_bvec<kVecInner>(B, A);
            if (rc == SEM_OK) rc = run_until_done(B, mode, maxit, need);
            if (rc == SEM_OK) rc = launch_bvec<kVecCorrect>(B, A);
            if (rc == SEM_OK) rc = launch_bax<double, double, 1>(B, B->grid_ax64);
            if (rc == SEM_OK) rc = launch_bvec<kVecResidual>(B, A);
        }
    }
    if (rc == SEM_OK) rc = launch_bvec<kVecCopyOut>(B, A);
    if (rc != SEM_OK) return rc;
    // per-problem results
    std::vector<BatchProb> hp(n);
    std::vector<CgState> hs(n);
    rc = cuda_check(cudaMemcpyAsync(hp.data(), B->d_probs, sizeof(BatchProb) * n, cudaMemcpyDeviceToHost, stream()),
                    "batch: results");
    for (int k = 0; k < n && rc == SEM_OK; ++k)
        rc = cuda_check(cudaMemcpyAsync(&hs[k], mode == 0 ? B->probs[k]->st : B->probs[k]->st_in, sizeof(CgState),
                                        cudaMemcpyDeviceToHost, stream()), "batch: results");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc != SEM_OK) return rc;
    for (int k = 0; k < n; ++k) {
        if (mode == 0) {
            iters[k] = hs[k].iter;
            res[k] = hs[k].rho0 > 0.0 ? std::sqrt(hs[k].rho / hs[k].rho0) : 0.0;
        } else {
            iters[k] = hp[k].inner_total;
            res[k] = hp[k].res;
        }
    }
    return SEM_OK;
}

}  // namespace sem
