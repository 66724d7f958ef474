// sem_ax.cu -- the local spectral-element Poisson operator ("ax", the most
// expensive kernel of the Nekbone CG iteration, Section VIII-B), FP64.
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
// Geometric factors are stored interleaved per node (48 bytes) and loaded as
// three 16-byte vectors, so a warp reads 1536 contiguous bytes per k-plane.
// N is a compile-time template parameter (the paper fixes N at code-generation
// time through its "jit" clause, Section VIII-B).
//
// CG variant (fused prologue/epilogue): p = r + beta p is formed on the staged
// slabs and written back, w = A_local p is stored, and the block's partial
// of sum_e p_e . w_e goes to a deterministic last-block reduction that also
// computes alpha = rho / <p, A p>.  Because p is continuous and masked,
// sum_e p_e^T A_e p_e equals p^T A p of the assembled masked operator.
#include <cuda_runtime.h>

#include <cstdio>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

struct AxParams {
    const double *x;    // plain: input x     CG: r
    double *y;          // plain: output y    CG: w
    double *p;          // CG: search direction (old in, new out)
    const double *G;    // [nL][6]
    double *partials;
    CgState *st;
    int32_t *status;
    int64_t E;
    double D[kMaxQ * kMaxQ];
};

template <int NQ, int EPB>
struct AxShape {
    static constexpr int NQ2 = NQ * NQ;
    static constexpr int NP = NQ2 * NQ;
    static constexpr int NTA = NQ2 * EPB;                 // threads with a column
    static constexpr int NT = (NTA + 31) / 32 * 32;       // threads launched
    static constexpr int SLAB = ((EPB * NP + 2) + 1) & ~1; // doubles per region (+16 B slack)
    static constexpr size_t SMEM = 16 + 3 * size_t(SLAB) * sizeof(double);
};

template <int NQ, int EPB, bool CG>
__global__ void __launch_bounds__(AxShape<NQ, EPB>::NT)
ax_f64_kernel(const AxParams P) {
    using S = AxShape<NQ, EPB>;
    constexpr int NQ2 = S::NQ2, NP = S::NP;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    double *regA = reinterpret_cast<double *>(smem + 16);
    double *regB = regA + S::SLAB;
    double *regC = regB + S::SLAB;

    if (CG && P.st->done) return;  // solve finished: the rest of the graph is a no-op

    const int tid = threadIdx.x;
    const int64_t e0 = int64_t(blockIdx.x) * EPB;
    const int ne = int(min(int64_t(EPB), P.E - e0));
    const uint32_t bytes = uint32_t(ne) * NP * uint32_t(sizeof(double));

    // ---- stage the slab(s): TMA for the aligned middle, plain loads for the edges
    const double *src1 = P.x + e0 * NP;                 // x (plain) or r (CG)
    const double *src2 = CG ? P.p + e0 * NP : nullptr;  // p (CG)
    double *s1 = slab_dst(regA, src1);
    double *s2 = CG ? slab_dst(regB, src2) : nullptr;
    const SlabPlan pl1 = slab_plan(src1, bytes);
    SlabPlan pl2{0, 0, 0};
    if (CG) pl2 = slab_plan(src2, bytes);
    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar, pl1.mid_bytes + pl2.mid_bytes);
        slab_issue(s1, src1, pl1, bar);
        if (CG) slab_issue(s2, src2, pl2, bar);
    }
    slab_edges(s1, src1, pl1, tid, S::NT);
    if (CG) slab_edges(s2, src2, pl2, tid, S::NT);
    const bool ok = mbar_wait_bounded(bar, 0, P.status);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, 0, nullptr);  // let copies in flight land before exit
        return;
    }

    const int eb = tid / NQ2;
    const int ij = tid - eb * NQ2;
    const int i = ij % NQ, j = ij / NQ;
    const bool act = (tid < S::NTA) && (eb < ne);
    const int64_t nb = (e0 + eb) * NP;  // first local node of this thread's element

    double xk[NQ];
    if (CG) {
        const double beta = P.st->beta;
        if (act) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const int q = eb * NP + k * NQ2 + ij;
                const double pn = fma(beta, s2[q], s1[q]);
                s2[q] = pn;
                xk[k] = pn;
                P.p[nb + k * NQ2 + ij] = pn;
            }
        }
        __syncthreads();
    } else if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) xk[k] = s1[eb * NP + k * NQ2 + ij];
    }
    const double *sx = (CG ? s2 : s1) + eb * NP;
    double *s_wr = (CG ? regA : regB) + eb * NP;
    double *s_ws = regC + eb * NP;

    double Di[NQ], Dj[NQ], Dti[NQ], Dtj[NQ];
#pragma unroll
    for (int l = 0; l < NQ; ++l) {
        Di[l] = P.D[i * NQ + l];
        Dj[l] = P.D[j * NQ + l];
        Dti[l] = P.D[l * NQ + i];
        Dtj[l] = P.D[l * NQ + j];
    }

    // ---- gradient in reference coordinates, then the geometric factors
    double wt[NQ];
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            double ur = 0.0, us = 0.0, ut = 0.0;
#pragma unroll
            for (int l = 0; l < NQ; ++l) {
                ur = fma(Di[l], sx[k * NQ2 + j * NQ + l], ur);
                us = fma(Dj[l], sx[k * NQ2 + l * NQ + i], us);
                ut = fma(P.D[k * NQ + l], xk[l], ut);
            }
            const double2 *g = reinterpret_cast<const double2 *>(P.G + 6 * (nb + k * NQ2 + ij));
            const double2 g01 = __ldg(g), g23 = __ldg(g + 1), g45 = __ldg(g + 2);
            // (rr, rs, rt, ss, st, tt) = (g01.x, g01.y, g23.x, g23.y, g45.x, g45.y)
            s_wr[k * NQ2 + ij] = g01.x * ur + g01.y * us + g23.x * ut;
            s_ws[k * NQ2 + ij] = g01.y * ur + g23.y * us + g45.x * ut;
            wt[k] = g23.x * ur + g45.x * us + g45.y * ut;
        }
    }
    __syncthreads();

    // ---- transposed derivatives, summed over the three directions
    double acc = 0.0;
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            double yv = 0.0;
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(Dti[l], s_wr[k * NQ2 + j * NQ + l], yv);
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(Dtj[l], s_ws[k * NQ2 + l * NQ + i], yv);
#pragma unroll
            for (int l = 0; l < NQ; ++l) yv = fma(P.D[l * NQ + k], wt[l], yv);
            P.y[nb + k * NQ2 + ij] = yv;
            if (CG) acc = fma(xk[k], yv, acc);
        }
    }
    if (CG) {
        const double bs = block_sum(acc, red);
        if (publish_partial(bs, P.partials, &P.st->ticket_ax)) {
            const double pap = finish_partials(P.partials, int(gridDim.x), &P.st->ticket_ax, red);
            if (tid == 0) {
                P.st->pap = pap;
                P.st->alpha = P.st->rho / pap;
            }
        }
    }
}

// Elements per block for each order: about 128 threads per block.
template <int NQ>
struct AxEpb {
    static constexpr int value = NQ <= 2 ? 32 : NQ == 3 ? 14 : NQ == 4 ? 8 : NQ == 5 ? 5
                               : NQ == 6 ? 3 : NQ <= 8 ? 2 : NQ == 9 ? 3 : 2;
};

// Opt the kernel in to its dynamic shared memory (once per process; done
// before any stream capture, from prepare_ax at problem set-up).
template <int NQ, bool CG>
static int ax_attr() {
    constexpr int EPB = AxEpb<NQ>::value;
    using S = AxShape<NQ, EPB>;
    static bool attr_set = false;
    if (!attr_set) {
        const int rc = cuda_check(cudaFuncSetAttribute(ax_f64_kernel<NQ, EPB, CG>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM)),
                                  "ax: smem attribute");
        if (rc != SEM_OK) return rc;
        attr_set = true;
    }
    return SEM_OK;
}

template <int NQ, bool CG>
static int launch_ax_nq(const Problem *Pb, const AxParams &a) {
    constexpr int EPB = AxEpb<NQ>::value;
    using S = AxShape<NQ, EPB>;
    auto kern = ax_f64_kernel<NQ, EPB, CG>;
    const int arc = ax_attr<NQ, CG>();
    if (arc != SEM_OK) return arc;
    const int64_t blocks = (Pb->E + EPB - 1) / EPB;
    if (CG && blocks > kMaxPartials) return set_error(SEM_ERANGE, "ax: too many elements for one launch");
    kern<<<unsigned(blocks), S::NT, S::SMEM, stream()>>>(a);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax_f64_kernel");
}

template <bool CG>
static int launch_ax_dispatch(const Problem *Pb, const AxParams &a) {
    switch (Pb->nq) {
        case 2: return launch_ax_nq<2, CG>(Pb, a);
        case 3: return launch_ax_nq<3, CG>(Pb, a);
        case 4: return launch_ax_nq<4, CG>(Pb, a);
        case 5: return launch_ax_nq<5, CG>(Pb, a);
        case 6: return launch_ax_nq<6, CG>(Pb, a);
        case 7: return launch_ax_nq<7, CG>(Pb, a);
        case 8: return launch_ax_nq<8, CG>(Pb, a);
        case 9: return launch_ax_nq<9, CG>(Pb, a);
        case 10: return launch_ax_nq<10, CG>(Pb, a);
        default: return set_error(SEM_EARG, "ax: unsupported order");
    }
}

template <int NQ>
static int prepare_nq() {
    const int rc = ax_attr<NQ, false>();
    return rc != SEM_OK ? rc : ax_attr<NQ, true>();
}

int prepare_ax(const Problem *Pb) {
    switch (Pb->nq) {
        case 2: return prepare_nq<2>();
        case 3: return prepare_nq<3>();
        case 4: return prepare_nq<4>();
        case 5: return prepare_nq<5>();
        case 6: return prepare_nq<6>();
        case 7: return prepare_nq<7>();
        case 8: return prepare_nq<8>();
        case 9: return prepare_nq<9>();
        case 10: return prepare_nq<10>();
        default: return set_error(SEM_EARG, "ax: unsupported order");
    }
}

static AxParams ax_params(const Problem *Pb) {
    AxParams a{};
    a.G = Pb->G;
    a.E = Pb->E;
    a.status = status_word();
    a.partials = Pb->partials;
    a.st = Pb->st;
    for (int q = 0; q < Pb->nq * Pb->nq; ++q) a.D[q] = Pb->oc.D[q];
    return a;
}

int launch_ax(const Problem *Pb, const double *x, double *y) {
    AxParams a = ax_params(Pb);
    a.x = x;
    a.y = y;
    return launch_ax_dispatch<false>(Pb, a);
}

int launch_ax_cg(const Problem *Pb) {
    AxParams a = ax_params(Pb);
    a.x = Pb->r;
    a.y = Pb->w;
    a.p = Pb->p;
    return launch_ax_dispatch<true>(Pb, a);
}

}  // namespace sem
