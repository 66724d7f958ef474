// sem_ax_kernel.cuh -- the local spectral-element Poisson operator ("ax", the
// most expensive kernel of the Nekbone CG iteration, Section VIII-B),
// templated on the arithmetic type T (double, or float for the inner solves
// of mixed-precision refinement) and on the storage type GT of the geometric
// factors (double, float or bf16).
//
// Per element e and node (i, j, k), with D the GLL derivative matrix and G the
// six symmetric geometric factors of the node:
//   u_r = sum_l D_il u_ljk,  u_s = sum_l D_jl u_ilk,  u_t = sum_l D_kl u_ijl
//   (w_r, w_s, w_t) = G (u_r, u_s, u_t)
//   y_ijk = sum_l D_li w_r,ljk + sum_l D_lj w_s,ilk + sum_l D_lk w_t,ijl
//
// GB300 mapping.  The paper's pattern maps the element loop to blockIdx.x and
// the three 1d-dof loops to threadIdx.{x,y,z} (Section III).  Here a block
// holds EPB elements and one thread per (i, j) column of an element; the
// k-line of the column lives in registers, so the t-direction sums need no
// shared memory.  The element's slab (x, or r and p in the CG variant) is
// staged in shared memory by the TMA engine (cp.async.bulk, completion on an
// mbarrier with a bounded wait); the r- and s-direction sums read it there.
// Geometric factors are stored interleaved per node and loaded as three
// vectors (16-byte double2, 8-byte float2, or 4-byte bf16 pairs), so a warp
// reads one contiguous run per k-plane.  N is a compile-time template
// parameter (the paper fixes N at code-generation time through its "jit"
// clause, Section VIII-B).
//
// CG variant (fused prologue/epilogue): p = r + beta p is formed on the staged
// slabs and written back, w = A_local p is stored, and the block's partial
// of sum_e p_e . w_e goes to a deterministic last-block reduction (FP64) that
// also computes alpha = rho / <p, A p>.  Because p is continuous and masked,
// sum_e p_e^T A_e p_e equals p^T A p of the assembled masked operator.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

template <typename T, typename GT>
struct AxArgs {
    const T *x;         // plain: input x     CG: r
    T *y;               // plain: output y    CG: w
    T *p;               // CG: search direction (old in, new out)
    const GT *G;        // [nL][6]
    double *partials;
    CgState *st;
    int32_t *status;
    const T *dinv;      // PCG: Jacobi inverse diagonal
    T *xs;              // CG: solution, updated x += alpha p_old before p is replaced
                        // (the previous iteration's x update, deferred); nullptr: none
    int64_t E;
    T D[kMaxQ * kMaxQ];
};

__device__ __forceinline__ void load_g6(const double *G, int64_t node, double (&g)[6]) {
    const double2 *q = reinterpret_cast<const double2 *>(G + 6 * node);
    const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    g[0] = a.x; g[1] = a.y; g[2] = b.x; g[3] = b.y; g[4] = c.x; g[5] = c.y;
}

__device__ __forceinline__ void load_g6(const float *G, int64_t node, float (&g)[6]) {
    const float2 *q = reinterpret_cast<const float2 *>(G + 6 * node);
    const float2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    g[0] = a.x; g[1] = a.y; g[2] = b.x; g[3] = b.y; g[4] = c.x; g[5] = c.y;
}

__device__ __forceinline__ float2 bf16x2_to_float2(unsigned v) {
    // a bf16 is the upper half of a float: widening is exact
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}

__device__ __forceinline__ void load_g6(const __nv_bfloat16 *G, int64_t node, float (&g)[6]) {
    const unsigned *q = reinterpret_cast<const unsigned *>(G + 6 * node);
    const float2 a = bf16x2_to_float2(__ldg(q)), b = bf16x2_to_float2(__ldg(q + 1)),
                 c = bf16x2_to_float2(__ldg(q + 2));
    g[0] = a.x; g[1] = a.y; g[2] = b.x; g[3] = b.y; g[4] = c.x; g[5] = c.y;
}

// The six factors of one node from shared memory (staged copies).
__device__ __forceinline__ void load_g6_smem(const __nv_bfloat16 *g, float (&v)[6]) {
    const unsigned *q = reinterpret_cast<const unsigned *>(g);
    const float2 a = bf16x2_to_float2(q[0]), b = bf16x2_to_float2(q[1]), c = bf16x2_to_float2(q[2]);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

__device__ __forceinline__ void load_g6_smem(const float *g, float (&v)[6]) {
    const float2 *q = reinterpret_cast<const float2 *>(g);
    const float2 a = q[0], b = q[1], c = q[2];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
}

template <int NQ, int EPB, typename T>
struct AxShape {
    static constexpr int NQ2 = NQ * NQ;
    static constexpr int NP = NQ2 * NQ;
    static constexpr int NTA = NQ2 * EPB;                 // threads with a column
    static constexpr int NT = (NTA + 31) / 32 * 32;       // threads launched
    static constexpr int VPQ = 16 / int(sizeof(T));       // values per 16 bytes
    static constexpr int SLAB = (EPB * NP + 2 * VPQ + VPQ - 1) / VPQ * VPQ;  // + 16 B slack, 16 B multiple
    static constexpr size_t SMEM = 16 + 3 * size_t(SLAB) * sizeof(T);
};

// One group of ne (<= EPB) elements starting at element e0, for a block of
// AxShape<NQ, EPB, T>::NT threads.  regA: 16-byte aligned shared memory of
// 3 * SLAB values; bar: an initialised mbarrier whose next completion is
// phase `phase`; D: the NQ x NQ derivative matrix (anything indexable).
// Returns false if the slab copy timed out (status set, copies drained).  In
// CG mode, *part receives this thread's partial of <p, A_local p> (in T).
template <int NQ, int EPB, typename T, typename GT, bool CG, typename DSrc, bool PRE = false>
__device__ __forceinline__ bool ax_group(const T *x, T *y, T *p, const GT *G, const DSrc &D, T beta,
                                         int64_t e0, int ne, T *regA, uint64_t *bar, uint32_t phase,
                                         int32_t *status, T *part, const T *dinv = nullptr, T *xs = nullptr,
                                         T xalpha = T(0)) {
    using S = AxShape<NQ, EPB, T>;
    constexpr int NQ2 = S::NQ2, NP = S::NP;
    T *regB = regA + S::SLAB;
    T *regC = regB + S::SLAB;
    const int tid = threadIdx.x;
    const uint32_t bytes = uint32_t(ne) * NP * uint32_t(sizeof(T));

    // ---- stage the slab(s): TMA for the aligned middle, plain loads for the edges
    const T *src1 = x + e0 * NP;                 // x (plain) or r (CG)
    const T *src2 = CG ? p + e0 * NP : nullptr;  // p (CG)
    T *s1 = slab_dst(regA, src1);
    T *s2 = CG ? slab_dst(regB, src2) : nullptr;
    const SlabPlan pl1 = slab_plan(src1, bytes);
    SlabPlan pl2{0, 0, 0};
    if (CG) pl2 = slab_plan(src2, bytes);
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, pl1.mid_bytes + pl2.mid_bytes);
        slab_issue(s1, src1, pl1, bar);
        if (CG) slab_issue(s2, src2, pl2, bar);
    }
    slab_edges(s1, src1, pl1, tid, S::NT);
    if (CG) slab_edges(s2, src2, pl2, tid, S::NT);
    const bool ok = mbar_wait_bounded(bar, phase, status);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, phase, nullptr);  // let copies in flight land before leaving
        return false;
    }

    const int eb = tid / NQ2;
    const int ij = tid - eb * NQ2;
    const int i = ij % NQ, j = ij / NQ;
    const bool act = (tid < S::NTA) && (eb < ne);
    const int64_t nb = (e0 + eb) * NP;  // first local node of this thread's element

    T xk[NQ];
    if (CG) {
        if (act) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const int q = eb * NP + k * NQ2 + ij;
                // PCG: p = M^-1 r + beta p with the Jacobi M
                const T zq = PRE ? dinv[nb + k * NQ2 + ij] * s1[q] : s1[q];
                if (xs) xs[nb + k * NQ2 + ij] = fma(xalpha, s2[q], xs[nb + k * NQ2 + ij]);
                const T pn = fma(beta, s2[q], zq);
                s2[q] = pn;
                xk[k] = pn;
                p[nb + k * NQ2 + ij] = pn;
            }
        }
        __syncthreads();
    } else if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) xk[k] = s1[eb * NP + k * NQ2 + ij];
    }
    const T *sx = (CG ? s2 : s1) + eb * NP;
    T *s_wr = (CG ? regA : regB) + eb * NP;
    T *s_ws = regC + eb * NP;

    T Di[NQ], Dj[NQ], Dti[NQ], Dtj[NQ];
#pragma unroll
    for (int l = 0; l < NQ; ++l) {
        Di[l] = D[i * NQ + l];
        Dj[l] = D[j * NQ + l];
        Dti[l] = D[l * NQ + i];
        Dtj[l] = D[l * NQ + j];
    }

    // ---- gradient in reference coordinates, then the geometric factors
    T wt[NQ];
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            T ur = T(0), us = T(0), ut = T(0);
#pragma unroll
            for (int l = 0; l < NQ; ++l) {
                ur = fma(Di[l], sx[k * NQ2 + j * NQ + l], ur);
                us = fma(Dj[l], sx[k * NQ2 + l * NQ + i], us);
                ut = fma(D[k * NQ + l], xk[l], ut);
            }
            T g[6];  // (rr, rs, rt, ss, st, tt)
            load_g6(G, nb + k * NQ2 + ij, g);
            s_wr[k * NQ2 + ij] = g[0] * ur + g[1] * us + g[2] * ut;
            s_ws[k * NQ2 + ij] = g[1] * ur + g[3] * us + g[4] * ut;
            wt[k] = g[2] * ur + g[4] * us + g[5] * ut;
        }
    }
    __syncthreads();

    // ---- transposed derivatives, summed over the three directions
    T acc = T(0);
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            T yv = T(0);
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(Dti[l], s_wr[k * NQ2 + j * NQ + l], yv);
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(Dtj[l], s_ws[k * NQ2 + l * NQ + i], yv);
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(D[l * NQ + k], wt[l], yv);
            y[nb + k * NQ2 + ij] = yv;
            if (CG) acc = fma(xk[k], yv, acc);
        }
    }
    if (CG) *part = acc;
    return true;
}

// Indexes the derivative matrix held in the kernel parameters.
template <typename T, typename GT>
struct ParamD {
    const AxArgs<T, GT> &a;
    __device__ __forceinline__ T operator[](int q) const { return a.D[q]; }
};

template <int NQ, int EPB, typename T, typename GT, bool CG, bool PRE = false>
__global__ void __launch_bounds__(AxShape<NQ, EPB, T>::NT)
ax_kernel(const AxArgs<T, GT> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *regA = reinterpret_cast<T *>(smem + 16);

    if (CG && P.st->done) return;  // solve finished: the rest of the graph is a no-op

    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    const int64_t e0 = int64_t(blockIdx.x) * EPB;
    const int ne = int(min(int64_t(EPB), P.E - e0));
    const T beta = CG ? T(P.st->beta) : T(0);
    const T xalpha = CG ? T(P.st->alpha) : T(0);   // read before this launch's last block replaces it
    T part = T(0);
    const ParamD<T, GT> D{P};
    if (!ax_group<NQ, EPB, T, GT, CG, ParamD<T, GT>, PRE>(P.x, P.y, P.p, P.G, D, beta, e0, ne, regA, bar, 0u,
                                                         P.status, &part, P.dinv, CG ? P.xs : nullptr, xalpha))
        return;
    if (CG) {
        // the column's partial is formed in T; the block and grid sums are FP64
        // (the grid sum over groups of blocks)
        const double bs = block_sum(double(part), red);
        if (publish_grouped(bs, P.partials, &P.st->ticket_ax)) {
            const double pap = finish_grouped(P.partials, &P.st->ticket_ax);
            if (threadIdx.x == 0) {
                P.st->pap = pap;
                P.st->alpha = P.st->rho / pap;
            }
        }
    }
}

// Elements per block: ~128 threads for FP64 (register bound), ~256 for FP32.
template <int NQ, typename T>
struct AxEpb {
    static constexpr int f64 = NQ <= 2 ? 32 : NQ == 3 ? 14 : NQ == 4 ? 8 : NQ == 5 ? 5
                             : NQ == 6 ? 3 : NQ <= 8 ? 2 : NQ == 9 ? 3 : 2;
    static constexpr int f32 = NQ <= 2 ? 64 : NQ == 3 ? 28 : NQ == 4 ? 16 : NQ == 5 ? 10
                             : NQ == 6 ? 7 : NQ == 7 ? 5 : NQ == 8 ? 4 : NQ == 9 ? 3 : 2;
    static constexpr int value = sizeof(T) == 8 ? f64 : f32;
};

template <int NQ, typename T, typename GT, bool CG, bool PRE = false>
static int ax_attr() {
    constexpr int EPB = AxEpb<NQ, T>::value;
    using S = AxShape<NQ, EPB, T>;
    static bool attr_set = false;
    if (!attr_set) {
        const int rc = cuda_check(cudaFuncSetAttribute(ax_kernel<NQ, EPB, T, GT, CG, PRE>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM)),
                                  "ax: smem attribute");
        if (rc != SEM_OK) return rc;
        attr_set = true;
    }
    return SEM_OK;
}

template <int NQ, typename T, typename GT, bool CG, bool PRE = false>
static int launch_ax_nq(const Problem *Pb, const AxArgs<T, GT> &a) {
    constexpr int EPB = AxEpb<NQ, T>::value;
    using S = AxShape<NQ, EPB, T>;
    const int arc = ax_attr<NQ, T, GT, CG, PRE>();
    if (arc != SEM_OK) return arc;
    const int64_t blocks = (Pb->E + EPB - 1) / EPB;
    if (CG && blocks > Pb->partials_cap) return set_error(SEM_ERANGE, "ax: more blocks than reduction slots");
    ax_kernel<NQ, EPB, T, GT, CG, PRE><<<unsigned(blocks), S::NT, S::SMEM, stream()>>>(a);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax_kernel");
}

template <typename T, typename GT, bool CG, bool PRE = false>
static int launch_ax_any(const Problem *Pb, const AxArgs<T, GT> &a) {
    switch (Pb->nq) {
        case 2: return launch_ax_nq<2, T, GT, CG, PRE>(Pb, a);
        case 3: return launch_ax_nq<3, T, GT, CG, PRE>(Pb, a);
        case 4: return launch_ax_nq<4, T, GT, CG, PRE>(Pb, a);
        case 5: return launch_ax_nq<5, T, GT, CG, PRE>(Pb, a);
        case 6: return launch_ax_nq<6, T, GT, CG, PRE>(Pb, a);
        case 7: return launch_ax_nq<7, T, GT, CG, PRE>(Pb, a);
        case 8: return launch_ax_nq<8, T, GT, CG, PRE>(Pb, a);
        case 9: return launch_ax_nq<9, T, GT, CG, PRE>(Pb, a);
        case 10: return launch_ax_nq<10, T, GT, CG, PRE>(Pb, a);
        default: return set_error(SEM_EARG, "ax: unsupported order");
    }
}

template <typename T, typename GT>
static int prepare_ax_any(const Problem *Pb) {
    int rc = SEM_OK;
    switch (Pb->nq) {
#define SEM_PREP(Q)                                      \
    case Q:                                              \
        rc = ax_attr<Q, T, GT, false>();                 \
        if (rc == SEM_OK) rc = ax_attr<Q, T, GT, true, true>();   \
        return rc != SEM_OK ? rc : ax_attr<Q, T, GT, true>();
        SEM_PREP(2) SEM_PREP(3) SEM_PREP(4) SEM_PREP(5) SEM_PREP(6)
        SEM_PREP(7) SEM_PREP(8) SEM_PREP(9) SEM_PREP(10)
#undef SEM_PREP
        default: return set_error(SEM_EARG, "ax: unsupported order");
    }
}

template <typename T, typename GT>
static AxArgs<T, GT> ax_args(const Problem *Pb, const GT *G, double *partials, CgState *st) {
    AxArgs<T, GT> a{};
    a.G = G;
    a.E = Pb->E;
    a.status = status_word();
    a.partials = partials;
    a.st = st;
    for (int q = 0; q < Pb->nq * Pb->nq; ++q) a.D[q] = T(Pb->oc.D[q]);
    return a;
}

}  // namespace sem
