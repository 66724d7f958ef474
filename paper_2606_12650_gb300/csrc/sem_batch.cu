// sem_batch.cu -- many independent Poisson problems of different sizes and
// orders solved together: each CG phase is a few persistent launches over all
// problems (one per order present for the operator, one for the vector
// update), replayed from a CUDA graph.
//
// Work lists.  Every problem is cut into operator items (~16384 local nodes:
// several passes of a 256-thread block) and vector items (row-aligned runs of
// ~16384 local nodes).  A persistent kernel's CTAs take items from a global
// counter (dynamic load balance across problems of very different cost).
// The operator list keeps each order's items together, and each order has
// its own kernel, compiled for that order and body with the body inlined;
// the vector kernel switches on N on the device.  The operator body and the
// elements per pass follow the per-order tuner's table for the batch's
// precision: the line body (sem_ax_lines.cuh), in double-word arithmetic for
// FP64 batches where the table chose that variant (sem_ax_dw.cuh), or the
// column body, passes of 256 / (N+1)^2 elements.  Items of problems whose
// solve finished are dropped from the lists between rounds (the items of one
// problem stay together and in order, so its reductions never change).
//
// Per-problem reductions.  Each item writes one partial (fixed-order block
// tree) to its own slot; the problem's last item to finish (per-problem
// ticket) sums the problem's slots in item order.  The items of a problem and
// the trees inside them do not depend on which other problems share the
// batch, so a problem's iterates are bit-identical alone or in any mix.
//
// States.  Each problem has its own CG state (and an inner one for mixed
// precision) and a few flags: `init` (start its solve this round), `refine`
// (mixed precision: its inner solve ended, so the FP64 correction, residual
// and restart run this round), `finished`.  Problems can join between rounds
// (continuous batching); finished ones are reported through a device list and
// their items leave the lists.  One round = the init phase for joining
// problems, K CG iterations replayed from a CUDA graph, and (mixed) the
// refinement phase for problems whose inner solve stopped -- each problem
// refines as soon as its own inner solve ends, not in lockstep.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "sem_ax_dw.cuh"
#include "sem_box.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kBatchThreads = 256;
constexpr int kVecItemNodes = 16384;
constexpr int kAxItemNodes = 16384;  // local nodes per operator item (several passes of the block)

struct BatchProb {
    int nq, nx, ny, nz;
    BoxDims bd;                     // the box with its fast divisors
    int64_t E, nL;
    const double *G;
    const float *Gdw;               // double-word factors (FP64 batches with the double-word body)
    const __nv_bfloat16 *G16;
    const float *G32;
    double *x, *r, *p, *w;          // FP64 CG vectors / refinement x, r
    float *d32, *r32, *p32, *w32;   // inner (FP32) CG vectors
    CgState *st, *st_in;
    const double *b;                // right-hand side
    int ax_first, ax_count;         // operator items
    int vec_first, vec_count;       // vector items
    int32_t init;                   // host sets: start this problem's solve next round
    int32_t refine;                 // mixed: inner solve ended, refine this round
    int32_t outer_done;             // mixed: true residual reached tol (or out of steps)
    int32_t finished;               // solve over; reported once in the finished list
    int32_t inner_total;            // mixed: inner iterations so far
    int32_t outer_steps;            // mixed: refinement steps so far
    double bb;                      // <b, b>
    double res;                     // mixed: current true relative residual
};

struct BatchItem {
    int prob, nq;
    int64_t first;  // first element (operator) or first local node (vector)
    int count;      // elements or nodes
    int group;      // operator items: elements per pass of the line body; 0 = column body
    int dw;         // operator items of FP64 batches: the line body in double-word arithmetic
};

struct BatchQueue {
    unsigned next, exited, pad0, pad1;
};

enum BatchQ : int { kQAx = 0, kQVec = 1, kNumQ = 2 };

// Operator bodies of a batch: every member of one order takes the same one.
enum AxBody : int { kBodyColumns = 0, kBodyLines = 1, kBodyDW = 2, kBodyNone = -1 };
constexpr int kOrders = kMaxQ - 1;  // N+1 = 2 .. kMaxQ

struct BatchCtl {
    BatchQueue q[kNumQ];            // [kQVec]: the vector phases' queue
    unsigned n_finished;            // entries in the finished list
    int n_items[kNumQ];             // items in the current (compacted) lists
    unsigned pad;
    // the operator list holds the items of each order together (order N+1 =
    // 2 first); each order's launch takes its range through its own queue
    BatchQueue q_ax[kOrders];
    int ax_first[kOrders], ax_count[kOrders];
    // the vector list likewise, for the per-order update launches
    int vec_first[kOrders], vec_count[kOrders];
    BatchQueue q_vec[kOrders];
};

struct Batch {
    int mode = 0;                   // 0 FP64 CG, 1 mixed (BF16 G), 2 mixed (FP32 G)
    int K = 16;                     // CG iterations per round
    double tol = 1e-8, inner_tol = 1e-3;
    int maxit = 100000, max_outer = 50;
    std::vector<Problem *> probs;
    int n_ax = 0, n_vec = 0;        // items in the device lists now
    // every member's items as built by batch_set, with its range in them; a
    // member whose solve finished is left out of the device lists (`gone`)
    std::vector<BatchItem> ax_all, vec_all;
    std::vector<int> ax_first_all, ax_count_all, vec_first_all, vec_count_all;
    int ord_body[kOrders];          // operator body per order (kBodyNone: no member of that order)
    int ord_count[kOrders];         // operator items per order in the device list now
    int ord_vcount[kOrders];        // vector items per order in the device list now
    int ord_res[kOrders] = {};      // resident CTAs of the order's operator and update kernels
    int ord_vres[kOrders] = {};
    std::vector<uint8_t> gone;
    int cap_probs = 0, cap_ax = 0, cap_vec = 0;
    BatchProb *d_probs = nullptr;
    BatchItem *d_ax = nullptr, *d_vec = nullptr;
    double *part = nullptr;         // one slot per operator item
    double *part_vec = nullptr;     // one slot per vector item (an order's update may run beside
                                    // another order's operator)
    int cap_part = 0, cap_part_vec = 0;
    uint32_t *tickets = nullptr;    // per problem: [ax, vec]
    int32_t *finished_ids = nullptr;
    BatchCtl *ctl = nullptr;
    BatchCtl *ctl_host = nullptr;
    unsigned seen_finished = 0;
    bool any_init = false;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
    // the buffers the captured round reads and its grids; the graph stays
    // valid while the buffers stay in place and the grids stay the same
    // (membership changes only rewrite the lists' contents and counts)
    const void *graph_bufs[7] = {};
    int graph_items[2] = {0, 0};    // power-of-two ceilings of the item counts at capture
    int ord_ranges[4 * kOrders];    // host copy of the device per-order ranges (operator, vector)
    int graph_ord[2 * kOrders] = {};  // per order: the captured launches' grid ceilings and body (0: none)
    int64_t graph_launches = 0;     // kernel launches in one replay
    // side streams and events that fork the per-order operator launches into
    // parallel branches of the captured round (the tail of one order's launch
    // overlaps the others)
    cudaStream_t side[kOrders] = {};
    cudaEvent_t fork = nullptr, join[kOrders] = {};
};

template <int NQ>
struct BEpb {
    static constexpr int value = kBatchThreads / (NQ * NQ);
};

// Dynamic shared memory of one order's operator body: the column body's
// slabs, or the line body's three regions (FP64-sized for the double-word
// body, whose values are FP32 pairs).
template <int NQ, typename T, int BODY>
inline size_t batch_ax_smem() {
    return BODY == kBodyColumns ? AxShape<NQ, BEpb<NQ>::value, T>::SMEM
                                : LineShape::smem(NQ, BEpb<NQ>::value, BODY == kBodyDW ? 8 : int(sizeof(T)));
}

// Derivative matrices of every order in constant memory: D depends only on
// N, so inside the switch case for order N every index is a compile-time
// constant and the products read constant-bank operands directly.
__constant__ double c_D64[kMaxQ - 1][kMaxQ * kMaxQ];
__constant__ float c_D32[kMaxQ - 1][kMaxQ * kMaxQ];
// even-odd coefficients of D ([0]) and D^T ([1]) for the line body
__constant__ EoMat<double> c_E64[kMaxQ - 1][2];
__constant__ EoMat<float> c_E32[kMaxQ - 1][2];
__constant__ EoMatDW c_EDW[kMaxQ - 1][2];

template <typename T>
__device__ __forceinline__ const EoMat<T> &const_eo(int nq, int which);
template <>
__device__ __forceinline__ const EoMat<double> &const_eo<double>(int nq, int which) { return c_E64[nq - 2][which]; }
template <>
__device__ __forceinline__ const EoMat<float> &const_eo<float>(int nq, int which) { return c_E32[nq - 2][which]; }

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
// One item of order NQ: `count` elements from `first`, taken in groups of
// what one pass of the block holds (`group` elements), so that an item's
// fixed costs -- the queue ticket, the block reduction of its partial -- are
// shared by several groups.  Each order and body has its own kernel, with
// the body inlined: as out-of-line calls from one kernel over all orders,
// the call convention's register saves and the caller's per-call-site
// stack spilled on every group.  *phase is the mbarrier phase of the next
// completion; each group uses one.
template <int NQ, typename T, typename GT, bool CG>
__device__ __forceinline__ bool batch_ax_item(const T *xin, T *yout, T *pv, const GT *G, T beta, int64_t first,
                                           int count, T *regA, uint64_t *bar, uint32_t *phase, int32_t *status,
                                           T *pt) {
    constexpr int GR = BEpb<NQ>::value;
    T acc = T(0);
    for (int g = 0; g < count; g += GR) {
        T part = T(0);
        const bool ok = ax_group<NQ, GR, T, GT, CG>(xin, yout, pv, G, ConstD<NQ, T>{}, beta, first + g,
                                                    min(GR, count - g), regA, bar, *phase, status, &part);
        *phase ^= 1u;
        if (!ok) return false;
        acc += part;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    *pt = acc;
    return true;
}

template <int NQ, typename T, typename GT, bool CG>
__device__ __forceinline__ bool batch_lines_item(const T *xin, T *yout, T *pv, const GT *G, T beta, int64_t first,
                                              int count, int group, T *regA, uint64_t *bar, uint32_t *phase,
                                              int32_t *status, T *pt) {
    constexpr int GM = kGLoad;   // factors loaded at use: the register prefetch would not fit 4 CTAs per SM
    T acc = T(0);
    for (int g = 0; g < count; g += group) {
        T part = T(0);
        const bool ok = lines_group<NQ, T, GT, CG, false, GM>(xin, yout, pv, G, const_eo<T>(NQ, 0),
                                                              const_eo<T>(NQ, 1), beta, T(0), nullptr, nullptr,
                                                              first + g, min(group, count - g), group, regA, bar,
                                                              *phase, status, &part);
        *phase ^= 1u;
        if (!ok) return false;
        acc += part;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    *pt = acc;
    return true;
}

// The double-word line body (FP64 batches): same passes as batch_lines_item.
template <int NQ, bool CG>
__device__ __forceinline__ bool batch_dw_item(const double *xin, double *yout, double *pv, const float *Gdw, double beta,
                                           int64_t first, int count, int group, double *regA, uint64_t *bar,
                                           uint32_t *phase, int32_t *status, double *pt) {
    double acc = 0.0;
    for (int g = 0; g < count; g += group) {
        double part = 0.0;
        const bool ok = lines_group_dw<NQ, CG, false>(xin, yout, pv, Gdw, c_EDW[NQ - 2][0], c_EDW[NQ - 2][1], beta,
                                                      0.0, nullptr, nullptr, first + g, min(group, count - g), group,
                                                      regA, bar, *phase, status, &part);
        *phase ^= 1u;
        if (!ok) return false;
        acc += part;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
    }
    *pt = acc;
    return true;
}

// mode: 0 = FP64 CG (p = r + beta p, w = A p), 1 = FP64 plain (w = A x),
//       2 = FP32 inner CG on the FP32 vectors
// One order's items (N+1 = NQ), one body.  FP32 items are HBM-bound: 4 CTAs
// per SM (<= 64 registers) for latency hiding; FP64 items keep the FP64
// bodies' registers (2 CTAs per SM).
template <typename T, typename GT, int MODE, int NQ, int BODY>
__global__ void __launch_bounds__(kBatchThreads, sizeof(T) == 4 ? 4 : 2)
    batch_ax_kernel(BatchProb *probs, const BatchItem *items, double *part, uint32_t *tickets, BatchCtl *ctl,
                    int32_t *status) {
    constexpr bool CG = MODE != 1;
    static_assert(BODY != kBodyDW || std::is_same<T, double>::value, "the double-word body is FP64");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    __shared__ int s_item;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *regA = reinterpret_cast<T *>(smem + 16);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    uint32_t phase = 0;
    BatchQueue *q = &ctl->q_ax[NQ - 2];
    const int first = ctl->ax_first[NQ - 2];
    const int nitems = ctl->ax_count[NQ - 2];
    while (true) {
        const int k = next_item(q, &s_item);
        if (k >= nitems) break;
        const int it = first + k;
        const BatchItem item = items[it];
        BatchProb &P = probs[item.prob];
        CgState *st = MODE == 2 ? P.st_in : P.st;
        if (CG && (st->done || P.finished)) continue;
        if (MODE == 1 && !P.refine) continue;      // refinement residual: refining problems only
        const T beta = CG ? T(st->beta) : T(0);
        const T *xin;
        T *yout, *pv;
        if (MODE == 0) { xin = reinterpret_cast<const T *>(P.r); yout = reinterpret_cast<T *>(P.w); pv = reinterpret_cast<T *>(P.p); }
        else if (MODE == 1) { xin = reinterpret_cast<const T *>(P.x); yout = reinterpret_cast<T *>(P.w); pv = nullptr; }
        else { xin = reinterpret_cast<const T *>(P.r32); yout = reinterpret_cast<T *>(P.w32); pv = reinterpret_cast<T *>(P.p32); }
        T pt = T(0);
        bool ok;
        if constexpr (BODY == kBodyDW)
            ok = batch_dw_item<NQ, CG>(xin, yout, pv, P.Gdw, beta, item.first, item.count, item.group, regA, bar,
                                       &phase, status, &pt);
        else if constexpr (BODY == kBodyLines)
            ok = batch_lines_item<NQ, T, GT, CG>(xin, yout, pv, prob_G<GT>(P), beta, item.first, item.count,
                                                 item.group, regA, bar, &phase, status, &pt);
        else
            ok = batch_ax_item<NQ, T, GT, CG>(xin, yout, pv, prob_G<GT>(P), beta, item.first, item.count, regA, bar,
                                              &phase, status, &pt);
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
    kVecInit64 = 2,     // joining problems: x = 0, p = 0, r = b, <b,b>
    kVecInner = 3,      // joining or refining problems: r32 = r, d32 = p32 = 0, inner state
    kVecCorrect = 4,    // refining problems: x += d32
    kVecResidual = 5,   // refining problems: r = b - mask(QQ^T w), <r,r>, outer test
};

struct VecArgs {
    int mode;           // solve kind (0 FP64 CG, 1/2 mixed)
    int maxit;          // CG (or inner CG) iteration limit
    int max_outer;      // mixed: refinement step limit
    int pad;
    double tol;         // relative residual target
    double inner_tol;   // mixed: minimum inner reduction
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

// The CG update of one item (FP64 CG, or the FP32 inner CG), returning the
// block's threads' <r, r> partials.
template <int NQ, int MODE>
__device__ __forceinline__ double vec_update_item(BatchProb &P, CgState *st, int64_t first, int count) {
    using T = typename std::conditional<MODE == kVecUpdate64, double, float>::type;
    constexpr int V = UpdVec<NQ, T>::value;
    const BoxDims bd = P.bd;   // in registers for the whole item
    T *x = MODE == kVecUpdate64 ? reinterpret_cast<T *>(P.x) : reinterpret_cast<T *>(P.d32);
    T *r = MODE == kVecUpdate64 ? reinterpret_cast<T *>(P.r) : reinterpret_cast<T *>(P.r32);
    const T *p = MODE == kVecUpdate64 ? reinterpret_cast<const T *>(P.p) : reinterpret_cast<const T *>(P.p32);
    const T *w = MODE == kVecUpdate64 ? reinterpret_cast<const T *>(P.w) : reinterpret_cast<const T *>(P.w32);
    const T alpha = T(st->alpha);
    T a = T(0);
    for (int v = threadIdx.x; v < count / V; v += blockDim.x)
        update_vec<NQ, V, T, T>(x, r, p, w, int(first) + v * V, bd, alpha, a);
    return double(a);
}

template <int NQ, int MODE>
__device__ __noinline__ double vec_item_body(BatchProb &P, CgState *st, int64_t first, int count) {
    double acc = 0.0;
    const int tid = threadIdx.x;
    if (MODE == kVecUpdate64 || MODE == kVecUpdate32) {
        acc = vec_update_item<NQ, MODE>(P, st, first, count);
    } else if (MODE == kVecInit64) {
        // <b, b> over global nodes (each counted at its first copy)
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            const double bl = P.b[l];
            P.x[l] = 0.0;
            P.p[l] = 0.0;
            P.r[l] = bl;
            if (box_node<NQ>(int(l), P.nx, P.ny, P.nz).owner) acc = fma(bl, bl, acc);
        }
    } else if (MODE == kVecInner) {
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            const float f = __double2float_rn(P.r[l]);
            P.r32[l] = f;
            P.d32[l] = 0.f;
            P.p32[l] = 0.f;
            if (box_node<NQ>(int(l), P.nx, P.ny, P.nz).owner) acc += double(f) * double(f);
        }
    } else if (MODE == kVecCorrect) {
        for (int v = tid; v < count; v += blockDim.x) {
            const int64_t l = first + v;
            P.x[l] += double(P.d32[l]);
        }
    } else if (MODE == kVecResidual) {
        for (int v = tid; v < count; v += blockDim.x)
            acc += residual_node<NQ>(P.r, P.b, P.w, int(first) + v, P.nx, P.ny, P.nz);
    }
    return acc;
}

// Mark a problem finished and append it to the finished list (thread 0).
__device__ __forceinline__ void finish_problem(BatchProb &P, int prob, BatchCtl *ctl, int32_t *finished_ids) {
    if (P.finished) return;
    P.finished = 1;
    const unsigned k = atomicAdd(&ctl->n_finished, 1u);
    finished_ids[k] = prob;
}

__device__ __forceinline__ void init_state(CgState *st, double rho0, double tol, int maxit) {
    st->rho = rho0;
    st->rho0 = rho0;
    st->alpha = st->beta = st->pap = 0.0;
    st->tol = tol;
    st->hist = nullptr;
    st->iter = 0;
    st->maxit = maxit;
    st->done = (rho0 == 0.0 || maxit <= 0) ? 1 : 0;
    st->ticket_ax = 0;
    st->ticket_up = 0;
}

template <int MODE>
__global__ void __launch_bounds__(kBatchThreads, MODE == kVecUpdate32 ? 4 : 3) batch_vec_kernel(BatchProb *probs, const BatchItem *items,
                                                                  double *part, uint32_t *tickets, BatchCtl *ctl,
                                                                  int32_t *finished_ids, VecArgs A) {
    __shared__ double red[32];
    __shared__ int s_item;
    constexpr bool REDUCES = MODE != kVecCorrect;
    BatchQueue *q = &ctl->q[kQVec];
    const int nitems = ctl->n_items[kQVec];
    while (true) {
        const int it = next_item(q, &s_item);
        if (it >= nitems) break;
        const BatchItem item = items[it];
        BatchProb &P = probs[item.prob];
        CgState *st = (MODE == kVecUpdate32 || MODE == kVecInner) ? P.st_in : P.st;
        // which problems take part in this phase
        bool on;
        if (MODE == kVecUpdate64 || MODE == kVecUpdate32) on = !st->done && !P.finished;
        else if (MODE == kVecInit64) on = P.init != 0;
        else if (MODE == kVecInner) on = (P.init || P.refine) && !P.outer_done;
        else on = P.refine != 0;   // correct, residual
        if (!on) continue;
        double acc = 0.0;
        switch (item.nq) {
#define SEM_BV(Q)                                                  \
    case Q:                                                        \
        acc = vec_item_body<Q, MODE>(P, st, item.first, item.count); \
        break;
            SEM_BV(2) SEM_BV(3) SEM_BV(4) SEM_BV(5) SEM_BV(6) SEM_BV(7) SEM_BV(8) SEM_BV(9) SEM_BV(10)
#undef SEM_BV
            default: break;
        }
        if (!REDUCES) continue;
        const double bs = block_sum(acc, red);
        double tot;
        if (!item_partial(bs, part, it, &tickets[2 * item.prob + 1], P.vec_first, P.vec_count, red, &tot) ||
            threadIdx.x != 0)
            continue;
        if (MODE == kVecUpdate64 || MODE == kVecUpdate32) {
            cg_close_iteration(st, tot);
            if (MODE == kVecUpdate64 && st->done) finish_problem(P, item.prob, ctl, finished_ids);
        } else if (MODE == kVecInit64) {
            init_state(P.st, tot, A.mode == 0 ? A.tol : 0.0, A.maxit);
            if (A.mode != 0) P.st_in->done = 1;   // no inner solve until kVecInner starts one
            P.bb = tot;
            P.res = tot > 0.0 ? 1.0 : 0.0;
            P.outer_done = tot == 0.0 ? 1 : 0;
            P.inner_total = 0;
            P.outer_steps = 0;
            P.refine = 0;
            if (tot == 0.0) finish_problem(P, item.prob, ctl, finished_ids);
        } else if (MODE == kVecInner) {
            init_state(st, tot, fmin(0.5, fmax(A.inner_tol, 0.5 * A.tol / P.res)), A.maxit);
        } else if (MODE == kVecResidual) {
            P.inner_total += P.st_in->iter;
            P.outer_steps += 1;
            P.res = P.bb > 0.0 ? sqrt(tot / P.bb) : 0.0;
            if (P.res <= A.tol || P.outer_steps >= A.max_outer) {
                P.outer_done = 1;
                finish_problem(P, item.prob, ctl, finished_ids);
            }
        }
    }
    leave_queue(q);
}

// The CG update phase for one order's items (its range of the vector list),
// the body inlined like the operator's.
constexpr int kUpd32Blocks = 4;   // CTAs per SM of the FP32 update (<= 64 registers)
template <int MODE, int NQ>
__global__ void __launch_bounds__(kBatchThreads, MODE == kVecUpdate32 ? kUpd32Blocks : 3)
    batch_update_kernel(BatchProb *probs, const BatchItem *items, double *part, uint32_t *tickets, BatchCtl *ctl,
                        int32_t *finished_ids) {
    static_assert(MODE == kVecUpdate64 || MODE == kVecUpdate32, "update phases only");
    __shared__ double red[32];
    __shared__ int s_item;
    BatchQueue *q = &ctl->q_vec[NQ - 2];
    const int first = ctl->vec_first[NQ - 2];
    const int nitems = ctl->vec_count[NQ - 2];
    while (true) {
        const int k = next_item(q, &s_item);
        if (k >= nitems) break;
        const int it = first + k;
        const BatchItem item = items[it];
        BatchProb &P = probs[item.prob];
        CgState *st = MODE == kVecUpdate32 ? P.st_in : P.st;
        if (st->done || P.finished) continue;
        const double acc = vec_update_item<NQ, MODE>(P, st, item.first, item.count);
        const double bs = block_sum(acc, red);
        double tot;
        if (!item_partial(bs, part, it, &tickets[2 * item.prob + 1], P.vec_first, P.vec_count, red, &tot) ||
            threadIdx.x != 0)
            continue;
        cg_close_iteration(st, tot);
        if (MODE == kVecUpdate64 && st->done) finish_problem(P, item.prob, ctl, finished_ids);
    }
    leave_queue(q);
}

// Per-problem flag updates between phases (one thread per problem).
enum FlagOp : int { kFlagClearInit = 0, kFlagMarkRefine = 1, kFlagClearRefine = 2 };

__global__ void batch_flags_kernel(BatchProb *probs, int n, int op) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    BatchProb &P = probs[k];
    if (op == kFlagClearInit) P.init = 0;
    else if (op == kFlagMarkRefine) P.refine = (!P.finished && !P.outer_done && P.st_in->done) ? 1 : 0;
    else P.refine = 0;
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

// Grid of a persistent launch over n items: the resident CTAs, or fewer for
// few items -- the next power of two of n, so that a captured round stays
// valid while the item count changes within a factor of two (extra CTAs find
// the queue empty and leave).
static int items_grid(int resident, int n) {
    int p = 1;
    while (p < n && p < (1 << 30)) p <<= 1;
    return std::max(1, std::min(resident, p));
}

// One order's operator kernel: its shared-memory limit set and its
// resident CTAs computed on first use (batch_set, before any capture), then
// launched over a grid for `count` items.
template <typename T, typename GT, int MODE, int NQ, int BODY>
struct BaxLaunch {
    static int resident(int *out) {
        static int grid = 0;
        if (!grid) {
            const void *k = reinterpret_cast<const void *>(batch_ax_kernel<T, GT, MODE, NQ, BODY>);
            const size_t sm = batch_ax_smem<NQ, T, BODY>();
            int rc = cuda_check(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)),
                                "batch: shared-memory attribute");
            if (rc == SEM_OK) rc = batch_grid(k, sm, &grid);
            if (rc != SEM_OK) return rc;
        }
        *out = grid;
        return SEM_OK;
    }
    static int launch(Batch *B, int count) {
        int res = 0;
        const int rc = resident(&res);
        if (rc != SEM_OK) return rc;
        batch_ax_kernel<T, GT, MODE, NQ, BODY>
            <<<unsigned(items_grid(res, count)), kBatchThreads, batch_ax_smem<NQ, T, BODY>(), stream()>>>(
                B->d_probs, B->d_ax, B->part, B->tickets, B->ctl, status_word());
        count_launches(1);
        return cuda_check(cudaGetLastError(), "batch_ax_kernel");
    }
};

// Dispatch on the order and body (prepare only, or launch for `count`
// items).  The double-word body exists for FP64 CG batches only.
template <typename T, typename GT, int MODE, int NQ>
static int bax_order(Batch *B, int body, int count, bool launch, int *res) {
    int r = 0;
    if (!res) res = &r;
    switch (body) {
        case kBodyColumns:
            return launch ? BaxLaunch<T, GT, MODE, NQ, kBodyColumns>::launch(B, count)
                          : BaxLaunch<T, GT, MODE, NQ, kBodyColumns>::resident(res);
        case kBodyLines:
            return launch ? BaxLaunch<T, GT, MODE, NQ, kBodyLines>::launch(B, count)
                          : BaxLaunch<T, GT, MODE, NQ, kBodyLines>::resident(res);
        case kBodyDW:
            if constexpr (MODE == 0)
                return launch ? BaxLaunch<T, GT, MODE, NQ, kBodyDW>::launch(B, count)
                              : BaxLaunch<T, GT, MODE, NQ, kBodyDW>::resident(res);
            [[fallthrough]];
        default: return set_error(SEM_EARG, "batch: no such operator body for this precision");
    }
}

// launch: launch order nq's kernel over `count` items; otherwise prepare it
// and report its resident CTAs in *res.
template <typename T, typename GT, int MODE>
static int bax(Batch *B, int nq, int body, int count, bool launch, int *res = nullptr) {
    switch (nq) {
        case 2: return bax_order<T, GT, MODE, 2>(B, body, count, launch, res);
        case 3: return bax_order<T, GT, MODE, 3>(B, body, count, launch, res);
        case 4: return bax_order<T, GT, MODE, 4>(B, body, count, launch, res);
        case 5: return bax_order<T, GT, MODE, 5>(B, body, count, launch, res);
        case 6: return bax_order<T, GT, MODE, 6>(B, body, count, launch, res);
        case 7: return bax_order<T, GT, MODE, 7>(B, body, count, launch, res);
        case 8: return bax_order<T, GT, MODE, 8>(B, body, count, launch, res);
        case 9: return bax_order<T, GT, MODE, 9>(B, body, count, launch, res);
        case 10: return bax_order<T, GT, MODE, 10>(B, body, count, launch, res);
        default: return set_error(SEM_EARG, "batch: unsupported order");
    }
}

// One launch per order present (fn(o) launches order o on the current
// stream), in sequence, or (parallel) the first on the current stream and
// the others on side streams forked from it and joined back.
template <typename F>
static int launch_orders(Batch *B, bool parallel, F &&fn) {
    const cudaStream_t s = stream();
    bool first = true;
    // the fork point: what precedes the phase on the current stream
    int rc = parallel ? cuda_check(cudaEventRecord(B->fork, s), "batch: fork") : SEM_OK;
    for (int o = 0; o < kOrders && rc == SEM_OK; ++o) {
        if (B->ord_body[o] == kBodyNone) continue;
        if (!parallel || first) {
            rc = fn(o);
            first = false;
            continue;
        }
        rc = cuda_check(cudaStreamWaitEvent(B->side[o], B->fork, 0), "batch: fork");
        if (rc == SEM_OK) {
            StreamScope on(B->side[o]);
            rc = fn(o);
        }
        if (rc == SEM_OK) rc = cuda_check(cudaEventRecord(B->join[o], B->side[o]), "batch: join");
        if (rc == SEM_OK) rc = cuda_check(cudaStreamWaitEvent(s, B->join[o], 0), "batch: join");
    }
    return rc;
}

// The operator phase of one precision.
template <typename T, typename GT, int MODE>
static int launch_bax(Batch *B, bool parallel = false) {
    return launch_orders(B, parallel, [B](int o) {
        return bax<T, GT, MODE>(B, o + 2, B->ord_body[o], B->ord_count[o], true);
    });
}

// One order's update kernel: resident CTAs on first use, then launched.
template <int MODE, int NQ>
struct UpdLaunch {
    static int resident(int *out) {
        static int grid = 0;
        if (!grid) {
            const int rc = batch_grid(reinterpret_cast<const void *>(batch_update_kernel<MODE, NQ>), 0, &grid);
            if (rc != SEM_OK) return rc;
        }
        *out = grid;
        return SEM_OK;
    }
    static int launch(Batch *B, int count) {
        int res = 0;
        const int rc = resident(&res);
        if (rc != SEM_OK) return rc;
        batch_update_kernel<MODE, NQ><<<unsigned(items_grid(res, count)), kBatchThreads, 0, stream()>>>(
            B->d_probs, B->d_vec, B->part_vec, B->tickets, B->ctl, B->finished_ids);
        count_launches(1);
        return cuda_check(cudaGetLastError(), "batch_update_kernel");
    }
};

template <int MODE>
static int upd(Batch *B, int nq, int count, bool launch, int *res = nullptr) {
    int r = 0;
    if (!res) res = &r;
    switch (nq) {
#define SEM_UPD(Q) \
    case Q: return launch ? UpdLaunch<MODE, Q>::launch(B, count) : UpdLaunch<MODE, Q>::resident(res);
        SEM_UPD(2) SEM_UPD(3) SEM_UPD(4) SEM_UPD(5) SEM_UPD(6) SEM_UPD(7) SEM_UPD(8) SEM_UPD(9) SEM_UPD(10)
#undef SEM_UPD
        default: return set_error(SEM_EARG, "batch: unsupported order");
    }
}

// Side streams and events of the parallel operator phase (made once, outside
// any capture).
static int make_side_streams(Batch *B) {
    if (B->fork) return SEM_OK;
    int rc = cuda_check(cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming), "batch: event");
    for (int o = 0; o < kOrders && rc == SEM_OK; ++o) {
        rc = cuda_check(cudaStreamCreateWithFlags(&B->side[o], cudaStreamNonBlocking), "batch: stream");
        if (rc == SEM_OK) rc = cuda_check(cudaEventCreateWithFlags(&B->join[o], cudaEventDisableTiming), "batch: event");
    }
    return rc;
}

// Every operator kernel this batch's rounds launch, prepared before capture.
static int prepare_bax(Batch *B) {
    for (int o = 0; o < kOrders; ++o) {
        const int body = B->ord_body[o];
        if (body == kBodyNone) continue;
        int rc;
        if (B->mode == 0) {
            rc = bax<double, double, 0>(B, o + 2, body, 0, false, &B->ord_res[o]);
            if (rc == SEM_OK) rc = upd<kVecUpdate64>(B, o + 2, 0, false, &B->ord_vres[o]);
        } else {
            rc = B->mode == 1 ? bax<float, __nv_bfloat16, 2>(B, o + 2, body, 0, false, &B->ord_res[o])
                              : bax<float, float, 2>(B, o + 2, body, 0, false, &B->ord_res[o]);
            if (rc == SEM_OK) rc = bax<double, double, 1>(B, o + 2, body, 0, false);
            if (rc == SEM_OK) rc = upd<kVecUpdate32>(B, o + 2, 0, false, &B->ord_vres[o]);
        }
        if (rc != SEM_OK) return rc;
    }
    return SEM_OK;
}

// Resident CTAs of one vector phase's kernel (the phases differ in
// registers); computed once, before any capture (batch_attrs).
template <int MODE>
static int vec_grid(int *out) {
    static int grid = 0;
    if (!grid) {
        const int rc = batch_grid(reinterpret_cast<const void *>(batch_vec_kernel<MODE>), 0, &grid);
        if (rc != SEM_OK) return rc;
    }
    *out = grid;
    return SEM_OK;
}

template <int MODE>
static int launch_bvec(Batch *B) {
    const VecArgs A{B->mode, B->maxit, B->max_outer, 0, B->tol, B->inner_tol};
    int grid = 0;
    const int rcg = vec_grid<MODE>(&grid);
    if (rcg != SEM_OK) return rcg;
    const int g = items_grid(grid, B->n_vec);
    batch_vec_kernel<MODE><<<unsigned(g), kBatchThreads, 0, stream()>>>(B->d_probs, B->d_vec, B->part_vec, B->tickets,
                                                                       B->ctl, B->finished_ids, A);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "batch_vec_kernel");
}

static int launch_flags(Batch *B, int op) {
    const int n = int(B->probs.size());
    batch_flags_kernel<<<unsigned((n + 127) / 128), 128, 0, stream()>>>(B->d_probs, n, op);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "batch_flags_kernel");
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
        static EoMat<double> e64[kMaxQ - 1][2];
        static EoMat<float> e32[kMaxQ - 1][2];
        static EoMatDW edw[kMaxQ - 1][2];
        for (int N = 1; N <= kMaxQ - 1; ++N) {
            const int nq = N + 1;
            double Dt[kMaxQ * kMaxQ];
            for (int i = 0; i < nq; ++i)
                for (int l = 0; l < nq; ++l) Dt[i * nq + l] = h64[N - 1][l * nq + i];
            e64[N - 1][0] = eo_coefficients<double>(h64[N - 1], nq);
            e64[N - 1][1] = eo_coefficients<double>(Dt, nq);
            e32[N - 1][0] = eo_coefficients<float>(h64[N - 1], nq);
            e32[N - 1][1] = eo_coefficients<float>(Dt, nq);
            edw[N - 1][0] = eo_coefficients_dw(h64[N - 1], nq);
            edw[N - 1][1] = eo_coefficients_dw(Dt, nq);
        }
        int rc = cuda_check(cudaMemcpyToSymbol(c_D64, h64, sizeof h64), "batch: D table");
        if (rc == SEM_OK) rc = cuda_check(cudaMemcpyToSymbol(c_D32, h32, sizeof h32), "batch: D table");
        if (rc == SEM_OK) rc = cuda_check(cudaMemcpyToSymbol(c_E64, e64, sizeof e64), "batch: even-odd table");
        if (rc == SEM_OK) rc = cuda_check(cudaMemcpyToSymbol(c_E32, e32, sizeof e32), "batch: even-odd table");
        if (rc == SEM_OK) rc = cuda_check(cudaMemcpyToSymbol(c_EDW, edw, sizeof edw), "batch: even-odd table");
        if (rc != SEM_OK) return rc;
        done = true;
    }
    (void)B;
    int g = 0;
    int rc = vec_grid<kVecInit64>(&g);
    if (rc == SEM_OK) rc = vec_grid<kVecInner>(&g);
    if (rc == SEM_OK) rc = vec_grid<kVecCorrect>(&g);
    if (rc == SEM_OK) rc = vec_grid<kVecResidual>(&g);
    return rc;
}

template <typename X>
static int grow(X **buf, int *cap, int need) {
    if (need <= *cap && *buf) return SEM_OK;
    const int c = std::max(need, std::max(16, 2 * *cap));
    X *nb = static_cast<X *>(dev_alloc(sizeof(X) * size_t(c)));
    if (!nb) return SEM_ENOMEM;
    if (*buf) dev_free(*buf);
    *buf = nb;
    *cap = c;
    return SEM_OK;
}

static int read_ctl(Batch *B) {
    int rc = cuda_check(cudaMemcpyAsync(B->ctl_host, B->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, stream()),
                        "batch: control read");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc == SEM_OK) rc = poll_status();
    return rc;
}

// Per-order ranges of the operator and vector lists to the device (ord_first:
// the operator firsts, then the vector firsts; the caller syncs).
static int upload_order_ranges(Batch *B, const int *ord_first) {
    for (int o = 0; o < kOrders; ++o) {
        B->ord_ranges[o] = ord_first[o];
        B->ord_ranges[kOrders + o] = B->ord_count[o];
        B->ord_ranges[2 * kOrders + o] = ord_first[kOrders + o];
        B->ord_ranges[3 * kOrders + o] = B->ord_vcount[o];
    }
    static_assert(offsetof(BatchCtl, ax_count) == offsetof(BatchCtl, ax_first) + kOrders * sizeof(int) &&
                      offsetof(BatchCtl, vec_first) == offsetof(BatchCtl, ax_first) + 2 * kOrders * sizeof(int) &&
                      offsetof(BatchCtl, vec_count) == offsetof(BatchCtl, ax_first) + 3 * kOrders * sizeof(int),
                  "ranges are copied as one block");
    return cuda_check(cudaMemcpyAsync(B->ctl->ax_first, B->ord_ranges, sizeof B->ord_ranges, cudaMemcpyHostToDevice,
                                      stream()), "batch: order ranges");
}

// What a captured round's launches depend on: per order, its operator body
// and the two launches' grids (0: no launches).  A grid is the resident CTAs
// or, for fewer items, their power-of-two ceiling, so item counts can change
// a lot at large sizes without a new capture.
static void order_signature(const Batch *B, int *out) {
    for (int o = 0; o < kOrders; ++o) {
        const bool on = B->ord_body[o] != kBodyNone;
        out[o] = on ? 4 * items_grid(B->ord_res[o], B->ord_count[o]) + B->ord_body[o] + 1 : 0;
        out[kOrders + o] = on ? items_grid(B->ord_vres[o], B->ord_vcount[o]) : 0;
    }
}

// New item ranges of the members after a compaction (ax_first, ax_count,
// vec_first, vec_count per member; a finished member gets empty ranges).
__global__ void batch_relist_kernel(BatchProb *probs, const int4 *ranges, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int4 r = ranges[k];
    probs[k].ax_first = r.x;
    probs[k].ax_count = r.y;
    probs[k].vec_first = r.z;
    probs[k].vec_count = r.w;
}

// Device item lists with the items of the members still solving, in member
// order (a member's items keep their order, so its reductions -- partials in
// its item order -- are unchanged and its iterates stay bit-identical).
// Finished members' items would otherwise each cost a queue ticket and a
// state read per launch for the rest of the solve.
static int compact(Batch *B) {
    const int n = int(B->probs.size());
    std::vector<BatchItem> ax, vec;
    std::vector<int4> ranges(n, make_int4(0, 0, 0, 0));
    int ord_first[2 * kOrders];
    for (int o = 0; o < kOrders; ++o) {   // by order, members in order
        ord_first[o] = int(ax.size());
        ord_first[kOrders + o] = int(vec.size());
        for (int k = 0; k < n; ++k) {
            if (B->gone[k] || B->probs[k]->nq - 2 != o) continue;
            const int a0 = B->ax_first_all[k], na = B->ax_count_all[k];
            const int v0 = B->vec_first_all[k], nv = B->vec_count_all[k];
            ranges[k] = make_int4(int(ax.size()), na, int(vec.size()), nv);
            ax.insert(ax.end(), B->ax_all.begin() + a0, B->ax_all.begin() + a0 + na);
            vec.insert(vec.end(), B->vec_all.begin() + v0, B->vec_all.begin() + v0 + nv);
        }
        B->ord_count[o] = int(ax.size()) - ord_first[o];
        B->ord_vcount[o] = int(vec.size()) - ord_first[kOrders + o];
    }
    int rc = SEM_OK;
    int4 *d_ranges = static_cast<int4 *>(dev_alloc(sizeof(int4) * size_t(std::max(n, 1))));
    if (!d_ranges) return SEM_ENOMEM;
    rc = cuda_check(cudaMemcpyAsync(d_ranges, ranges.data(), sizeof(int4) * size_t(n), cudaMemcpyHostToDevice,
                                    stream()), "batch: ranges");
    if (rc == SEM_OK) {
        batch_relist_kernel<<<unsigned((n + 127) / 128), 128, 0, stream()>>>(B->d_probs, d_ranges, n);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "batch_relist_kernel");
    }
    if (rc == SEM_OK && !ax.empty())
        rc = cuda_check(cudaMemcpyAsync(B->d_ax, ax.data(), sizeof(BatchItem) * ax.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    if (rc == SEM_OK && !vec.empty())
        rc = cuda_check(cudaMemcpyAsync(B->d_vec, vec.data(), sizeof(BatchItem) * vec.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    const int counts[kNumQ] = {int(ax.size()), int(vec.size())};
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B->ctl->n_items, counts, sizeof counts, cudaMemcpyHostToDevice, stream()),
                        "batch: item counts");
    if (rc == SEM_OK) rc = upload_order_ranges(B, ord_first);
    // the host copies above come from pageable memory; finish them before
    // the vectors go out of scope
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    dev_free(d_ranges);
    if (rc == SEM_OK) {
        B->n_ax = counts[0];
        B->n_vec = counts[1];
    }
    return rc;
}

Batch *batch_new(int mode, double tol, int maxit, double inner_tol, int max_outer, int K) {
    Batch *B = new Batch();
    B->mode = mode;
    B->tol = tol;
    B->maxit = maxit;
    B->inner_tol = inner_tol;
    B->max_outer = max_outer;
    B->K = K;
    std::fill(B->ord_body, B->ord_body + kOrders, int(kBodyNone));
    std::fill(B->ord_count, B->ord_count + kOrders, 0);
    std::fill(B->ord_vcount, B->ord_vcount + kOrders, 0);
    return B;
}

// Set the problems of the batch.  Problems already in the batch keep their
// solve state; problems listed with start[k] != 0 (re)start their solve with
// right-hand side b[k] at the next round.  Invalidates the captured graph.
int batch_set(Batch *B, Problem **probs, const double *const *b, const uint8_t *start, int n) {
    int rc = SEM_OK;
    if (!B->ctl) {
        B->ctl = static_cast<BatchCtl *>(dev_alloc(sizeof(BatchCtl)));
        if (!B->ctl) return SEM_ENOMEM;
        rc = cuda_check(cudaMemsetAsync(B->ctl, 0, sizeof(BatchCtl), stream()), "batch: control");
        if (rc == SEM_OK) rc = cuda_check(cudaMallocHost(&B->ctl_host, sizeof(BatchCtl)), "batch: pinned");
        if (rc == SEM_OK) rc = batch_attrs(B);
        if (rc != SEM_OK) return rc;
    }
    // current device state of the members (to keep it for continuing problems)
    std::vector<BatchProb> old(B->probs.size());
    if (!old.empty()) {
        rc = cuda_check(cudaMemcpyAsync(old.data(), B->d_probs, sizeof(BatchProb) * old.size(),
                                        cudaMemcpyDeviceToHost, stream()), "batch: state read");
        if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
        if (rc != SEM_OK) return rc;
    }
    std::vector<BatchProb> hp(n);
    std::vector<BatchItem> ax, vec;
    std::vector<BatchItem> by_ord[kOrders];   // operator items of each order, members in order
    std::vector<BatchItem> by_ord_v[kOrders]; // vector items likewise
    int ord_body[kOrders];
    std::fill(ord_body, ord_body + kOrders, int(kBodyNone));
    bool any_init = false;
    for (int k = 0; k < n && rc == SEM_OK; ++k) {
        Problem *P = probs[k];
        if (B->mode != 0) rc = mixed_prepare(P, B->mode == 1 ? kGBF16 : kGF32);
        if (rc != SEM_OK) break;
        BatchProb &q = hp[k];
        memset(&q, 0, sizeof q);
        for (size_t j = 0; j < B->probs.size(); ++j)
            if (B->probs[j] == P) q = old[j];       // keep the solve state
        q.nq = P->nq; q.nx = P->nx; q.ny = P->ny; q.nz = P->nz;
        q.bd = box_dims(P->nx, P->ny, P->nz);
        q.E = P->E; q.nL = P->nL;
        q.G = P->G; q.G16 = static_cast<const __nv_bfloat16 *>(P->G16); q.G32 = static_cast<const float *>(P->G32);
        q.x = P->x; q.r = P->r; q.p = P->p; q.w = P->w;
        q.d32 = P->d32; q.r32 = P->r32; q.p32 = P->p32; q.w32 = P->w32;
        q.st = P->st; q.st_in = P->st_in ? P->st_in : P->st;
        if (start[k]) {
            q.b = b[k];
            q.init = 1;
            q.finished = 0;
            q.refine = 0;
            q.outer_done = 0;
            any_init = true;
        }
        // operator body from the tuner's table; a pass of the line body fills
        // the engine's fixed 256-thread CTA (the table's elements per block
        // size stand-alone blocks, whose count per SM varies with it); an
        // item holds several passes (~kAxItemNodes local nodes)
        const int full = kBatchThreads / (P->nq * P->nq);
        const TuneChoice c = tune_get(B->mode == 0 ? kTuneF64 : (B->mode == 1 ? kTuneF32G16 : kTuneF32G32), P->nq);
        // the double-word variant: its line body in FP64 batches (factors
        // made here, before any capture); mixed batches (whose FP64 operator
        // runs only for the refinement residual) keep the FP64 line body
        const bool dw = B->mode == 0 && c.variant == kAxLinesDW;
        if (dw) {
            rc = dw_prepare(P);
            if (rc != SEM_OK) break;
            q.Gdw = P->Gdw;
        }
        const bool lines = c.variant == kAxLines || c.variant == kAxLinesPrefetch || c.variant == kAxLinesStaged ||
                           c.variant == kAxLinesDW;
        const int group = full;
        const int np = P->nq * P->nq * P->nq;
        const int per_item = group * std::max(1, kAxItemNodes / (np * group));
        const int o = P->nq - 2;
        const int body = dw ? kBodyDW : (lines ? kBodyLines : kBodyColumns);
        if (ord_body[o] != kBodyNone && ord_body[o] != body) {
            rc = set_error(SEM_EARG, "batch: members of one order with different operator bodies");
            break;
        }
        ord_body[o] = body;
        std::vector<BatchItem> &oa = by_ord[o];
        q.ax_first = int(oa.size());   // within its order's items; placed below
        for (int64_t e = 0; e < P->E; e += per_item)
            oa.push_back(BatchItem{k, P->nq, e, int(std::min<int64_t>(per_item, P->E - e)), lines ? group : 0,
                                   dw ? 1 : 0});
        q.ax_count = int(oa.size()) - q.ax_first;
        const int64_t chunk = std::max<int64_t>(P->nq, (kVecItemNodes / P->nq) * P->nq);
        std::vector<BatchItem> &ov = by_ord_v[o];
        q.vec_first = int(ov.size());  // within its order's items; placed below
        for (int64_t l = 0; l < P->nL; l += chunk)
            ov.push_back(BatchItem{k, P->nq, l, int(std::min<int64_t>(chunk, P->nL - l)), 0});
        q.vec_count = int(ov.size()) - q.vec_first;
    }
    if (rc != SEM_OK) return rc;
    // the lists: each order's items together, orders ascending
    int ord_first[2 * kOrders];
    for (int o = 0; o < kOrders; ++o) {
        ord_first[o] = int(ax.size());
        ax.insert(ax.end(), by_ord[o].begin(), by_ord[o].end());
        ord_first[kOrders + o] = int(vec.size());
        vec.insert(vec.end(), by_ord_v[o].begin(), by_ord_v[o].end());
    }
    for (int k = 0; k < n; ++k) {
        hp[k].ax_first += ord_first[probs[k]->nq - 2];
        hp[k].vec_first += ord_first[kOrders + probs[k]->nq - 2];
    }
    std::copy(ord_body, ord_body + kOrders, B->ord_body);
    for (int o = 0; o < kOrders; ++o) {
        B->ord_count[o] = int(by_ord[o].size());
        B->ord_vcount[o] = int(by_ord_v[o].size());
    }
    rc = prepare_bax(B);
    if (rc == SEM_OK) rc = make_side_streams(B);
    if (rc != SEM_OK) return rc;
    const int cap_probs_before = B->cap_probs;
    rc = grow(&B->d_probs, &B->cap_probs, std::max(n, 1));
    if (rc == SEM_OK && (B->cap_probs != cap_probs_before || !B->tickets || !B->finished_ids)) {
        // tickets (2 per problem) and finished ids follow the problem capacity
        if (B->tickets) dev_free(B->tickets);
        if (B->finished_ids) dev_free(B->finished_ids);
        B->tickets = static_cast<uint32_t *>(dev_alloc(sizeof(uint32_t) * 2 * size_t(B->cap_probs)));
        B->finished_ids = static_cast<int32_t *>(dev_alloc(sizeof(int32_t) * (size_t(B->cap_probs) + 1)));
        if (!B->tickets || !B->finished_ids) rc = SEM_ENOMEM;
    }
    if (rc == SEM_OK) rc = grow(&B->d_ax, &B->cap_ax, std::max<int>(int(ax.size()), 1));
    if (rc == SEM_OK) rc = grow(&B->d_vec, &B->cap_vec, std::max<int>(int(vec.size()), 1));
    if (rc == SEM_OK) rc = grow(&B->part, &B->cap_part, B->cap_ax);
    if (rc == SEM_OK) rc = grow(&B->part_vec, &B->cap_part_vec, B->cap_vec);
    if (rc != SEM_OK) return rc;
    B->probs.assign(probs, probs + n);
    B->n_ax = int(ax.size());
    B->n_vec = int(vec.size());
    B->ax_all = ax;
    B->vec_all = vec;
    B->ax_first_all.assign(n, 0);
    B->ax_count_all.assign(n, 0);
    B->vec_first_all.assign(n, 0);
    B->vec_count_all.assign(n, 0);
    for (int k = 0; k < n; ++k) {
        B->ax_first_all[k] = hp[k].ax_first;
        B->ax_count_all[k] = hp[k].ax_count;
        B->vec_first_all[k] = hp[k].vec_first;
        B->vec_count_all[k] = hp[k].vec_count;
    }
    B->gone.assign(n, 0);
    B->any_init = any_init;
    if (n)
        rc = cuda_check(cudaMemcpyAsync(B->d_probs, hp.data(), sizeof(BatchProb) * n, cudaMemcpyHostToDevice,
                                        stream()), "batch: descriptors");
    if (rc == SEM_OK && !ax.empty())
        rc = cuda_check(cudaMemcpyAsync(B->d_ax, ax.data(), sizeof(BatchItem) * ax.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    if (rc == SEM_OK && !vec.empty())
        rc = cuda_check(cudaMemcpyAsync(B->d_vec, vec.data(), sizeof(BatchItem) * vec.size(), cudaMemcpyHostToDevice,
                                        stream()), "batch: items");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemsetAsync(B->tickets, 0, sizeof(uint32_t) * 2 * size_t(B->cap_probs), stream()), "batch");
    // the finished list restarts with the new membership
    if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(&B->ctl->n_finished, 0, sizeof(unsigned), stream()), "batch");
    const int counts[kNumQ] = {B->n_ax, B->n_vec};
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(B->ctl->n_items, counts, sizeof counts, cudaMemcpyHostToDevice, stream()),
                        "batch: item counts");
    if (rc == SEM_OK) rc = upload_order_ranges(B, ord_first);
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    B->seen_finished = 0;
    // the captured round reads the lists and counts from device memory: it
    // is captured again only if a buffer moved (grew)
    const void *bufs[7] = {B->d_probs, B->d_ax, B->d_vec, B->part, B->part_vec, B->tickets, B->finished_ids};
    int ord_now[2 * kOrders];
    order_signature(B, ord_now);
    const bool same_grids = std::equal(ord_now, ord_now + 2 * kOrders, B->graph_ord);
    if (B->graph && !(same_grids && std::equal(bufs, bufs + 7, B->graph_bufs))) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return rc;
}

void batch_destroy(Batch *B) {
    if (!B) return;
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (int o = 0; o < kOrders; ++o) {
        if (B->side[o]) cudaStreamDestroy(B->side[o]);
        if (B->join[o]) cudaEventDestroy(B->join[o]);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    void *ptrs[] = {B->d_probs, B->d_ax, B->d_vec, B->part, B->part_vec, B->tickets, B->finished_ids, B->ctl};
    for (void *q : ptrs)
        if (q) dev_free(q);
    if (B->ctl_host) cudaFreeHost(B->ctl_host);
    delete B;
}

int batch_size(const Batch *B) { return int(B->probs.size()); }
int64_t batch_total_nodes(const Batch *B) {
    int64_t t = 0;
    for (const Problem *P : B->probs) t += P->nL;
    return t;
}

// K iterations of (operator, update) for the batch's precision, captured once
// per membership.
static int capture(Batch *B) {
    if (B->graph && B->graph_stream == stream()) return SEM_OK;
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(stream(), cudaStreamCaptureModeThreadLocal), "batch: capture");
    if (rc != SEM_OK) return rc;
    int orders = 0;
    for (int o = 0; o < kOrders; ++o) orders += B->ord_body[o] != kBodyNone;
    // each order's problems are independent of the others': its K
    // iterations form one chain of (operator, update) launches, the orders'
    // chains parallel branches of the round
    rc = launch_orders(B, true, [B](int o) {
        const int nq = o + 2, body = B->ord_body[o], na = B->ord_count[o], nv = B->ord_vcount[o];
        int r = SEM_OK;
        for (int k = 0; k < B->K && r == SEM_OK; ++k) {
            if (B->mode == 0) {
                r = bax<double, double, 0>(B, nq, body, na, true);
                if (r == SEM_OK) r = upd<kVecUpdate64>(B, nq, nv, true);
            } else {
                r = B->mode == 1 ? bax<float, __nv_bfloat16, 2>(B, nq, body, na, true)
                                 : bax<float, float, 2>(B, nq, body, na, true);
                if (r == SEM_OK) r = upd<kVecUpdate32>(B, nq, nv, true);
            }
        }
        return r;
    });
    B->graph_launches = int64_t(B->K) * 2 * orders;
    count_launches(-B->graph_launches);
    const int rc_end = cuda_check(cudaStreamEndCapture(stream(), &g), "batch: end capture");
    if (rc == SEM_OK) rc = rc_end;
    if (rc == SEM_OK) rc = cuda_check(cudaGraphInstantiate(&B->graph, g, 0), "batch: instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc == SEM_OK) {
        B->graph_stream = stream();
        const void *bufs[7] = {B->d_probs, B->d_ax, B->d_vec, B->part, B->part_vec, B->tickets, B->finished_ids};
        std::copy(bufs, bufs + 7, B->graph_bufs);
        B->graph_items[0] = items_grid(1 << 30, B->n_ax);
        B->graph_items[1] = items_grid(1 << 30, B->n_vec);
        order_signature(B, B->graph_ord);
    }
    return rc;
}

// One round: start joining problems, K CG iterations, refinement of problems
// whose inner solve ended (mixed).  Appends the problems that finished during
// the round (indices into the member list) to *done.
int batch_round(Batch *B, std::vector<int> *done) {
    const int rc = batch_round_launch(B);
    return rc != SEM_OK ? rc : batch_round_finish(B, done);
}

// A round's launches (init for joining problems, K CG iterations, the
// refinement phases), issued on the library stream without waiting, so the
// host can prepare other work (the server admits requests) meanwhile.
int batch_round_launch(Batch *B) {
    if (B->probs.empty()) return SEM_OK;
    int rc = SEM_OK;
    if (B->any_init) {
        rc = launch_bvec<kVecInit64>(B);
        if (rc == SEM_OK && B->mode != 0) rc = launch_bvec<kVecInner>(B);
        if (rc == SEM_OK) rc = launch_flags(B, kFlagClearInit);
        B->any_init = false;
        if (rc != SEM_OK) return rc;
    }
    rc = capture(B);
    if (rc == SEM_OK) rc = cuda_check(cudaGraphLaunch(B->graph, stream()), "batch: graph launch");
    if (rc != SEM_OK) return rc;
    count_launches(B->graph_launches);
    if (B->mode != 0) {
        rc = launch_flags(B, kFlagMarkRefine);
        if (rc == SEM_OK) rc = launch_bvec<kVecCorrect>(B);
        if (rc == SEM_OK) rc = launch_bax<double, double, 1>(B);
        if (rc == SEM_OK) rc = launch_bvec<kVecResidual>(B);
        if (rc == SEM_OK) rc = launch_bvec<kVecInner>(B);
        if (rc == SEM_OK) rc = launch_flags(B, kFlagClearRefine);
        if (rc != SEM_OK) return rc;
    }
    return SEM_OK;
}

// Waits for the round and reports the problems that finished in it.
int batch_round_finish(Batch *B, std::vector<int> *done) {
    if (B->probs.empty()) return SEM_OK;
    int rc = read_ctl(B);
    if (rc != SEM_OK) return rc;
    const unsigned nf = B->ctl_host->n_finished;
    if (nf > B->seen_finished) {
        std::vector<int32_t> ids(nf - B->seen_finished);
        rc = cuda_check(cudaMemcpyAsync(ids.data(), B->finished_ids + B->seen_finished, sizeof(int32_t) * ids.size(),
                                        cudaMemcpyDeviceToHost, stream()), "batch: finished list");
        if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
        if (rc != SEM_OK) return rc;
        for (int32_t k : ids) {
            done->push_back(k);
            if (k >= 0 && k < int(B->gone.size())) B->gone[k] = 1;
        }
        B->seen_finished = nf;
        rc = compact(B);
        if (rc != SEM_OK) return rc;
    }
    return SEM_OK;
}

// Per-problem results after the problem finished: iterations (CG, or inner
// iterations for mixed) and the relative residual (recursive for CG, true
// for mixed).
int batch_results(Batch *B, int64_t *iters, double *res) {
    const int n = batch_size(B);
    std::vector<BatchProb> hp(n);
    std::vector<CgState> hs(n);
    int rc = cuda_check(cudaMemcpyAsync(hp.data(), B->d_probs, sizeof(BatchProb) * n, cudaMemcpyDeviceToHost,
                                        stream()), "batch: results");
    for (int k = 0; k < n && rc == SEM_OK; ++k)
        rc = cuda_check(cudaMemcpyAsync(&hs[k], B->probs[k]->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                        "batch: results");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc != SEM_OK) return rc;
    for (int k = 0; k < n; ++k) {
        if (B->mode == 0) {
            iters[k] = hs[k].iter;
            res[k] = hs[k].rho0 > 0.0 ? std::sqrt(hs[k].rho / hs[k].rho0) : 0.0;
        } else {
            iters[k] = hp[k].inner_total;
            res[k] = hp[k].res;
        }
    }
    return SEM_OK;
}

// The same for the listed members only (a server retiring a few of many).
int batch_results_of(Batch *B, const std::vector<int> &which, int64_t *iters, double *res) {
    const size_t m = which.size();
    std::vector<BatchProb> hp(m);
    std::vector<CgState> hs(m);
    int rc = SEM_OK;
    for (size_t j = 0; j < m && rc == SEM_OK; ++j) {
        const int k = which[j];
        if (k < 0 || k >= batch_size(B)) return set_error(SEM_EARG, "batch: member index out of range");
        rc = cuda_check(cudaMemcpyAsync(&hp[j], B->d_probs + k, sizeof(BatchProb), cudaMemcpyDeviceToHost, stream()),
                        "batch: results");
        if (rc == SEM_OK)
            rc = cuda_check(cudaMemcpyAsync(&hs[j], B->probs[k]->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                            "batch: results");
    }
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc != SEM_OK) return rc;
    for (size_t j = 0; j < m; ++j) {
        if (B->mode == 0) {
            iters[j] = hs[j].iter;
            res[j] = hs[j].rho0 > 0.0 ? std::sqrt(hs[j].rho / hs[j].rho0) : 0.0;
        } else {
            iters[j] = hp[j].inner_total;
            res[j] = hp[j].res;
        }
    }
    return SEM_OK;
}

// Fixed batch: every problem starts now; rounds until all have finished.
int batch_solve(Batch *B, const double *b_all, double *x_all, double tol, int maxit, int mode, double inner_tol,
                int max_outer, int64_t *iters, double *res) {
    if (mode < 0 || mode > 2) return set_error(SEM_EARG, "batch_solve: mode must be 0 (fp64), 1 (bf16), 2 (fp32)");
    if (maxit < 1) return set_error(SEM_EARG, "batch_solve: maxit must be >= 1");
    const int n = batch_size(B);
    if (mode != B->mode && B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    B->mode = mode;
    B->tol = tol;
    B->maxit = maxit;
    B->inner_tol = inner_tol;
    B->max_outer = max_outer;
    std::vector<Problem *> ps = B->probs;
    std::vector<const double *> bs(n);
    std::vector<uint8_t> start(n, 1);
    int64_t off = 0;
    for (int k = 0; k < n; ++k) {
        bs[k] = b_all + off;
        off += ps[k]->nL;
    }
    int rc = batch_set(B, ps.data(), bs.data(), start.data(), n);
    std::vector<int> done;
    // enough rounds for every problem's iteration limits
    const int64_t per_solve = mode == 0 ? int64_t(maxit) : int64_t(maxit + 1) * std::max(1, max_outer);
    const int64_t max_rounds = per_solve / std::max(1, B->K) + max_outer + 4;
    for (int64_t round = 0; round < max_rounds && rc == SEM_OK && int(done.size()) < n; ++round)
        rc = batch_round(B, &done);
    if (rc != SEM_OK) return rc;
    off = 0;
    for (int k = 0; k < n && rc == SEM_OK; ++k) {
        rc = cuda_check(cudaMemcpyAsync(x_all + off, ps[k]->x, sizeof(double) * ps[k]->nL, cudaMemcpyDeviceToDevice,
                                        stream()), "batch: copy x");
        off += ps[k]->nL;
    }
    if (rc != SEM_OK) return rc;
    return batch_results(B, iters, res);
}

int batch_create(Problem **probs, int n, Batch **out) {
    *out = nullptr;
    if (n < 1) return set_error(SEM_EARG, "batch: needs at least one problem");
    Batch *B = batch_new(0, 1e-8, 100000, 1e-3, 50, 16);
    int64_t tot = 0;
    for (int k = 0; k < n; ++k) tot += probs[k]->nL;
    B->K = tot < (int64_t(1) << 22) ? 32 : 16;
    std::vector<const double *> bs(n, nullptr);
    std::vector<uint8_t> start(n, 0);
    // prepare both mixed precisions up front so later solves need no allocation
    int rc = SEM_OK;
    for (int k = 0; k < n && rc == SEM_OK; ++k) {
        rc = mixed_prepare(probs[k], kGBF16);
        if (rc == SEM_OK) rc = mixed_prepare(probs[k], kGF32);
    }
    if (rc == SEM_OK) rc = batch_set(B, probs, bs.data(), start.data(), n);
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "batch: sync");
    if (rc != SEM_OK) {
        batch_destroy(B);
        return rc;
    }
    *out = B;
    return SEM_OK;
}

}  // namespace sem
