// sem_ax_lines.cuh -- the local Poisson operator with whole lines per thread
// and the even-odd split of the 1d derivative matrix.
//
// Same map as ax_kernel (sem_ax_kernel.cuh): per element and node
//   (u_r, u_s, u_t) = (D_r u, D_s u, D_t u),  w = G (u_r, u_s, u_t),
//   y = D_r^T w_r + D_s^T w_s + D_t^T w_t,
// but each thread applies a 1d matrix to a whole line of N+1 values at once,
// so the line can be split into its even and odd parts.  The GLL derivative
// matrix is centro-antisymmetric (D_{N-i,N-l} = -D_{il}, the nodes being
// symmetric about 0), and so is D^T; for such an M and u_e = u_l + u_{N-l},
// u_o = u_l - u_{N-l} (l < (N+1)/2),
//   (M u)_i     =  A_i + B_i,     (M u)_{N-i} = -A_i + B_i,
//   A_i = sum_l Me_il u_e,l (+ M_{i,h} u_h),   B_i = sum_l Mo_il u_o,l,
// with Me_il = (M_il + M_{i,N-l}) / 2, Mo_il = (M_il - M_{i,N-l}) / 2 and, for
// odd N+1, the middle node h = N/2 (whose own output is B_h).  For N+1 = 8 a
// line costs 48 operations instead of 64: on GB300, whose FP64 pipe is 1/64
// of the FP32 rate, the FP64 operator is bound by exactly this count.
//
// Thread roles (one thread per (a, b) in [0, N+1)^2 of its element):
//   r lines: row (j, k) = (a, b)      s lines: column (i, k) = (a, b)
//   t lines: (i, j) = (a, b), kept in registers (as in ax_kernel).
// Phases: (0) stage x (or r and p, forming p = r + beta p) in shared memory;
// (1) r and s lines of x into U and V, t line into registers; (2) per node
// (U, V, u_t) <- G (u_r, u_s, u_t); (3) transposed r and s lines in place,
// t line in registers; (4) y = (U + V) + y_t, stored, and <p, y> in CG mode.
// The number of elements per block is a launch parameter (tuned per N).
#pragma once

#include "sem_ax_kernel.cuh"

namespace sem {

// Even-odd coefficients of one centro-antisymmetric (N+1) x (N+1) matrix M.
// e[i*H + l], o[i*H + l] for i < H (and o row H for odd N+1), l < H;
// m[i] = M[i][h] (odd N+1 only); H = (N+1)/2 rounded down.
template <typename T>
struct EoMat {
    T e[25];
    T o[30];
    T m[5];
};

template <typename T, typename GT>
struct AxLineArgs {
    AxArgs<T, GT> a;
    EoMat<T> d;      // of D   (gradient)
    EoMat<T> dt;     // of D^T (divergence)
    int epb;         // elements per block
};

// y = M u by the even-odd split.
template <int NQ, typename T>
__device__ __forceinline__ void eo_apply(const T (&u)[NQ], T (&y)[NQ], const EoMat<T> &c) {
    constexpr int H = NQ / 2;
    constexpr bool ODD = (NQ & 1) != 0;
    T ue[H], uo[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        ue[l] = u[l] + u[NQ - 1 - l];
        uo[l] = u[l] - u[NQ - 1 - l];
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        T a = c.e[i * H] * ue[0];
        T b = c.o[i * H] * uo[0];
#pragma unroll
        for (int l = 1; l < H; ++l) {
            a = fma(c.e[i * H + l], ue[l], a);
            b = fma(c.o[i * H + l], uo[l], b);
        }
        if (ODD) a = fma(c.m[i], u[H], a);
        y[i] = a + b;
        y[NQ - 1 - i] = b - a;
    }
    if (ODD) {
        T b = c.o[H * H] * uo[0];
#pragma unroll
        for (int l = 1; l < H; ++l) b = fma(c.o[H * H + l], uo[l], b);
        y[H] = b;
    }
}

struct LineShape {
    // values per buffer for epb elements: + 2 x 16 B slack for the slab
    // alignment shift, rounded to 16 B
    template <typename T>
    static __host__ __device__ int slab(int np, int epb) {
        const int vpq = 16 / int(sizeof(T));
        return (epb * np + 2 * vpq + vpq - 1) / vpq * vpq;
    }
    template <typename T>
    static __host__ __device__ size_t smem(int np, int epb) {
        return 16 + 3 * size_t(slab<T>(np, epb)) * sizeof(T);
    }
};

template <int NQ, typename T, typename GT, bool CG, bool PRE>
__global__ void __launch_bounds__(512) ax_lines_kernel(const AxLineArgs<T, GT> P) {
    constexpr int NQ2 = NQ * NQ, NP = NQ2 * NQ;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    const AxArgs<T, GT> &A = P.a;
    if (CG && A.st->done) return;  // solve finished: the rest of the graph is a no-op

    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    const int SL = LineShape::slab<T>(NP, P.epb);
    T *regA = reinterpret_cast<T *>(smem + 16);
    T *regB = regA + SL;
    T *regC = regB + SL;
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int64_t e0 = int64_t(blockIdx.x) * P.epb;
    const int ne = int(min(int64_t(P.epb), A.E - e0));

    if (tid == 0) mbar_init(bar, 1);
    __syncthreads();

    // ---- (0) stage the slab(s): TMA for the aligned middle, plain loads for the edges
    const uint32_t bytes = uint32_t(ne) * NP * uint32_t(sizeof(T));
    const T *src1 = A.x + e0 * NP;                 // x (plain) or r (CG)
    const T *src2 = CG ? A.p + e0 * NP : nullptr;  // p (CG)
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
    slab_edges(s1, src1, pl1, tid, nthreads);
    if (CG) slab_edges(s2, src2, pl2, tid, nthreads);
    const bool ok = mbar_wait_bounded(bar, 0u, A.status);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, 0u, nullptr);  // let copies in flight land before leaving
        return;
    }

    const int eb = tid / NQ2;
    const int ab = tid - eb * NQ2;
    const int a = ab % NQ, b = ab / NQ;
    const bool act = eb < ne;
    const int64_t nb = (e0 + eb) * NP;
    const int rq = b * NQ2 + a * NQ;   // r line (j, k) = (a, b): first node
    const int cq = b * NQ2 + a;        // s line (i, k) = (a, b): first node, stride NQ
    const int tq = b * NQ + a;         // t line (i, j) = (a, b): first node, stride NQ2

    T xk[NQ];
    if (CG) {
        const T beta = T(A.st->beta);
        if (act) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const int q = eb * NP + k * NQ2 + tq;
                const T zq = PRE ? A.dinv[nb + k * NQ2 + tq] * s1[q] : s1[q];
                const T pn = fma(beta, s2[q], zq);
                s2[q] = pn;
                xk[k] = pn;
                A.p[nb + k * NQ2 + tq] = pn;
            }
        }
        __syncthreads();
    } else if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) xk[k] = s1[eb * NP + k * NQ2 + tq];
    }
    const T *SX = (CG ? s2 : s1) + eb * NP;
    T *SU = (CG ? regA : regB) + eb * NP;
    T *SV = regC + eb * NP;

    // ---- (1) gradient lines
    T ut[NQ];
    if (act) {
        T u[NQ], y[NQ];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SX[rq + l];
        eo_apply<NQ, T>(u, y, P.d);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SU[rq + l] = y[l];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SX[cq + l * NQ];
        eo_apply<NQ, T>(u, y, P.d);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SV[cq + l * NQ] = y[l];
        eo_apply<NQ, T>(xk, ut, P.d);
    }
    __syncthreads();

    // ---- (2) geometric factors, node by node
    T wt[NQ];
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int q = k * NQ2 + tq;
            const T ur = SU[q], us = SV[q];
            T g[6];
            load_g6(A.G, nb + q, g);
            SU[q] = g[0] * ur + g[1] * us + g[2] * ut[k];
            SV[q] = g[1] * ur + g[3] * us + g[4] * ut[k];
            wt[k] = g[2] * ur + g[4] * us + g[5] * ut[k];
        }
    }
    __syncthreads();

    // ---- (3) divergence lines (in place: each line has one owner)
    T yt[NQ];
    if (act) {
        T u[NQ], y[NQ];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SU[rq + l];
        eo_apply<NQ, T>(u, y, P.dt);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SU[rq + l] = y[l];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SV[cq + l * NQ];
        eo_apply<NQ, T>(u, y, P.dt);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SV[cq + l * NQ] = y[l];
        eo_apply<NQ, T>(wt, yt, P.dt);
    }
    __syncthreads();

    // ---- (4) sum of the three directions
    T acc = T(0);
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int q = k * NQ2 + tq;
            const T yv = (SU[q] + SV[q]) + yt[k];
            A.y[nb + q] = yv;
            if (CG) acc = fma(SX[q], yv, acc);
        }
    }
    if (CG) {
        // the thread's partial is formed in T; the block and grid sums are FP64
        const double bs = block_sum(double(acc), red);
        if (publish_partial(bs, A.partials, &A.st->ticket_ax)) {
            const double pap = finish_partials(A.partials, int(gridDim.x), &A.st->ticket_ax, red);
            if (tid == 0) {
                A.st->pap = pap;
                A.st->alpha = A.st->rho / pap;
            }
        }
    }
}

// Host: even-odd coefficients of M (row-major nq x nq), in FP64 then cast.
template <typename T>
inline EoMat<T> eo_coefficients(const double *M, int nq) {
    EoMat<T> c{};
    const int N = nq - 1, H = nq / 2;
    for (int i = 0; i < H; ++i)
        for (int l = 0; l < H; ++l) {
            c.e[i * H + l] = T(0.5 * (M[i * nq + l] + M[i * nq + N - l]));
            c.o[i * H + l] = T(0.5 * (M[i * nq + l] - M[i * nq + N - l]));
        }
    if (nq & 1) {
        for (int l = 0; l < H; ++l) c.o[H * H + l] = T(0.5 * (M[H * nq + l] - M[H * nq + N - l]));
        for (int i = 0; i < H; ++i) c.m[i] = T(M[i * nq + H]);
    }
    return c;
}

template <typename T, typename GT>
inline AxLineArgs<T, GT> line_args(const AxArgs<T, GT> &a, const double *D, int nq, int epb) {
    AxLineArgs<T, GT> L{};
    L.a = a;
    double Dt[kMaxQ * kMaxQ];
    for (int i = 0; i < nq; ++i)
        for (int l = 0; l < nq; ++l) Dt[i * nq + l] = D[l * nq + i];
    L.d = eo_coefficients<T>(D, nq);
    L.dt = eo_coefficients<T>(Dt, nq);
    L.epb = epb;
    return L;
}

// Threads of a block of epb elements (multiple of 32), or 0 if epb elements
// do not fit one block.
inline int line_threads(int nq, int epb) {
    const int t = (epb * nq * nq + 31) / 32 * 32;
    return t <= 512 ? t : 0;
}

template <int NQ, typename T, typename GT, bool CG, bool PRE>
static int launch_lines_nq(const Problem *Pb, const AxLineArgs<T, GT> &L) {
    constexpr int NP = NQ * NQ * NQ;
    const int nt = line_threads(NQ, L.epb);
    if (L.epb < 1 || nt == 0) return set_error(SEM_EARG, "ax lines: elements per block out of range");
    const size_t sm = LineShape::smem<T>(NP, L.epb);
    if (sm > size_t(227) * 1024) return set_error(SEM_EARG, "ax lines: shared memory per block too large");
    auto kern = ax_lines_kernel<NQ, T, GT, CG, PRE>;
    // raise the dynamic shared-memory limit when a larger block is first
    // asked for (the tuner and the first solve do so before any capture)
    static size_t sm_set = 0;
    if (sm > sm_set) {
        const int rc = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm)),
                                  "ax lines: smem attribute");
        if (rc != SEM_OK) return rc;
        sm_set = sm;
    }
    const int64_t blocks = (Pb->E + L.epb - 1) / L.epb;
    if (CG && blocks > kMaxPartials) return set_error(SEM_ERANGE, "ax lines: too many elements for one launch");
    kern<<<unsigned(blocks), nt, sm, stream()>>>(L);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax_lines_kernel");
}

template <typename T, typename GT, bool CG, bool PRE = false>
static int launch_lines_any(const Problem *Pb, const AxLineArgs<T, GT> &L) {
    switch (Pb->nq) {
        case 2: return launch_lines_nq<2, T, GT, CG, PRE>(Pb, L);
        case 3: return launch_lines_nq<3, T, GT, CG, PRE>(Pb, L);
        case 4: return launch_lines_nq<4, T, GT, CG, PRE>(Pb, L);
        case 5: return launch_lines_nq<5, T, GT, CG, PRE>(Pb, L);
        case 6: return launch_lines_nq<6, T, GT, CG, PRE>(Pb, L);
        case 7: return launch_lines_nq<7, T, GT, CG, PRE>(Pb, L);
        case 8: return launch_lines_nq<8, T, GT, CG, PRE>(Pb, L);
        case 9: return launch_lines_nq<9, T, GT, CG, PRE>(Pb, L);
        case 10: return launch_lines_nq<10, T, GT, CG, PRE>(Pb, L);
        default: return set_error(SEM_EARG, "ax lines: unsupported order");
    }
}

}  // namespace sem
