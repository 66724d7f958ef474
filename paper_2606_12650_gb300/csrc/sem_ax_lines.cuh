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
    // FP32: (e[i*H + l], o[i*H + l]) side by side, the operand pairs of the
    // packed two-lane sums (unused in FP64)
    alignas(8) T eo[sizeof(T) == 4 ? 50 : 2];
};

template <typename T, typename GT>
struct AxLineArgs {
    AxArgs<T, GT> a;
    EoMat<T> d;      // of D   (gradient)
    EoMat<T> dt;     // of D^T (divergence)
    int epb;         // elements per block
};

// FP32 and even N+1: the even and odd sums of row i advance together as one
// two-lane pair, (A_i, B_i) += (Me_il, Mo_il) (u_e,l, u_o,l), one packed
// f32x2 fma per term instead of two; each lane rounds like the scalar fma,
// so y is bit-identical to the scalar form.
template <int NQ>
__device__ __forceinline__ void eo_apply_x2(const float (&u)[NQ], float (&y)[NQ], const EoMat<float> &c) {
    constexpr int H = NQ / 2;
    float2 v[H];
#pragma unroll
    for (int l = 0; l < H; ++l) v[l] = make_float2(u[l] + u[NQ - 1 - l], u[l] - u[NQ - 1 - l]);
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float2 s = __fmul2_rn(make_float2(c.eo[2 * (i * H)], c.eo[2 * (i * H) + 1]), v[0]);
#pragma unroll
        for (int l = 1; l < H; ++l)
            s = __ffma2_rn(make_float2(c.eo[2 * (i * H + l)], c.eo[2 * (i * H + l) + 1]), v[l], s);
        y[i] = s.x + s.y;
        y[NQ - 1 - i] = s.y - s.x;
    }
}

// y = M u by the even-odd split.
template <int NQ, typename T>
__device__ __forceinline__ void eo_apply(const T (&u)[NQ], T (&y)[NQ], const EoMat<T> &c) {
    constexpr int H = NQ / 2;
    constexpr bool ODD = (NQ & 1) != 0;
    if constexpr (sizeof(T) == 4 && !ODD) {
        eo_apply_x2<NQ>(u, y, c);
        return;
    }
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

// In-register rotation v[m] <- v[(m - R) mod NQ] for a per-thread R
// (NQ a power of two): log2(NQ) stages of selects, no local memory.
template <int NQ, typename T>
__device__ __forceinline__ void rotate_right(T (&v)[NQ], int R) {
#pragma unroll
    for (int bit = 1; bit < NQ; bit <<= 1) {
        const bool on = (R & bit) != 0;
        T w[NQ];
#pragma unroll
        for (int m = 0; m < NQ; ++m) w[m] = on ? v[(m - bit) & (NQ - 1)] : v[m];
#pragma unroll
        for (int m = 0; m < NQ; ++m) v[m] = w[m];
    }
}

// Shared-memory layout.  The staged input slab(s) keep the global layout
// (TMA copies them as they are).  U and V, written and read only by this
// kernel, are padded for N+1 = 8: node (i, j, k) of an element at
// k P2 + j P1 + i with P1 = 9, P2 = 72, so the rows and the columns a warp
// touches at one step fall in distinct banks (FP32; two lanes per bank pair
// in FP64, the minimum for 8-byte values) -- unpadded, rows 32 B apart put
// 8 lanes on one bank.  Other orders keep the compact layout (measured:
// padding there costs more in occupancy than it saves in conflicts).
template <int NQ>
struct LinePad {
    static constexpr int P1 = NQ == 8 ? NQ + 1 : NQ, P2 = NQ * P1, NPP = NQ * P2;
};

// Where phase 2 gets the geometric factors: loaded from global memory at use
// (kGLoad), loaded into registers before the slab wait (kGRegs, BF16 only),
// or copied into shared memory by the TMA engine with the slab (kGStaged,
// FP32 arithmetic only: an element's FP64 factors would take 24 KB).
enum LineG : int { kGLoad = 0, kGRegs = 1, kGStaged = 2 };

struct LineShape {
    // values per buffer for epb elements: the larger of the staged slab
    // (+ 2 x 16 B slack for its alignment shift) and the padded U / V
    // layout, rounded to 16 B
    static __host__ __device__ int region(int nq, int epb, int elem_bytes) {
        const int vpq = 16 / elem_bytes;
        const int slab = epb * nq * nq * nq + 2 * vpq;
        const int pad = epb * nq * nq * (nq == 8 ? nq + 1 : nq);
        const int m = slab > pad ? slab : pad;
        return (m + vpq - 1) / vpq * vpq;
    }
    // bytes of the staged factors (g_bytes per node; 0 when not staged), + 32 B slack
    static __host__ __device__ size_t gstage(int nq, int epb, int g_bytes) {
        return g_bytes ? (size_t(epb) * nq * nq * nq * g_bytes + 32 + 15) / 16 * 16 : 0;
    }
    static __host__ __device__ size_t smem(int nq, int epb, int elem_bytes, int g_bytes = 0) {
        const size_t regions = 3 * size_t(region(nq, epb, elem_bytes)) * size_t(elem_bytes);
        // the regions also hold one double per thread for the block's final sum
        const size_t sums = size_t((epb * nq * nq + 31) / 32 * 32) * sizeof(double);
        return 16 + (regions > sums ? regions : sums) + gstage(nq, epb, g_bytes);
    }
};

// One group of ne (<= epb) elements starting at element e0, for a block of
// at least epb (N+1)^2 threads.  regA: 16-byte aligned shared memory of
// 3 LineShape::region(N+1, epb) values; bar: an initialised mbarrier whose
// next completion is phase `phase`; cd, ct: even-odd coefficients of D and
// D^T.  CG mode: p = r + beta p (PRE: M^-1 r + beta p), and xs += xalpha p_old
// first when xs is given; *part receives this thread's <p, A_local p> partial
// (in T).  Returns false if the slab copy timed out (status set, copies
// drained).
// GM (LineG): kGRegs loads the element's BF16 factors into registers (3
// words per node) before the slab wait, kGStaged has the TMA engine copy
// them into shared memory after the three regions, with the slab; either
// way their latency overlaps the slab copy instead of stalling phase 2.
template <int NQ, typename T, typename GT, bool CG, bool PRE, int GM>
__device__ __forceinline__ bool lines_group(const T *x, T *y, T *p, const GT *G, const EoMat<T> &cd,
                                            const EoMat<T> &ct, T beta, T xalpha, T *xs, const T *dinv, int64_t e0,
                                            int ne, int epb, T *regA, uint64_t *bar, uint32_t phase,
                                            int32_t *status, T *part) {
    constexpr bool PF = GM == kGRegs;
    constexpr bool GS = GM == kGStaged;
    static_assert(!PF || sizeof(GT) == 2, "G prefetch is for BF16 factors");
    static_assert(!GS || sizeof(T) == 4, "G staging is for FP32 arithmetic");
    constexpr int NQ2 = NQ * NQ, NP = NQ2 * NQ;
    constexpr int P1 = LinePad<NQ>::P1, P2 = LinePad<NQ>::P2, NPP = LinePad<NQ>::NPP;
    // N+1 = 8: the staged slab's rows and columns are read in a per-thread
    // rotated order (then rotated back in registers), so a warp's lanes hit
    // distinct banks: rows of 8 values start 32 B (FP32) or 64 B (FP64)
    // apart, 4 or 2 to a 128-byte bank row, hence the rotation by row / 4
    // or row / 2; columns of one warp differ in k, hence the rotation by k.
    constexpr bool ROT = NQ == 8;
    constexpr int RPB = sizeof(T) == 8 ? 2 : 4;
    const int RG = LineShape::region(NQ, epb, int(sizeof(T)));
    T *regB = regA + RG;
    T *regC = regB + RG;
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;

    // ---- (0) stage the slab(s): TMA for the aligned middle, plain loads for the edges
    const uint32_t bytes = uint32_t(ne) * NP * uint32_t(sizeof(T));
    const T *src1 = x + e0 * NP;                 // x (plain) or r (CG)
    const T *src2 = CG ? p + e0 * NP : nullptr;  // p (CG)
    T *s1 = slab_dst(regA, src1);
    T *s2 = CG ? slab_dst(regB, src2) : nullptr;
    const SlabPlan pl1 = slab_plan(src1, bytes);
    SlabPlan pl2{0, 0, 0};
    if (CG) pl2 = slab_plan(src2, bytes);
    // staged factors: the group's factors are one contiguous run
    const unsigned char *gsrc = reinterpret_cast<const unsigned char *>(G + 6 * e0 * NP);
    unsigned char *gdst = GS ? slab_dst(reinterpret_cast<unsigned char *>(regC + RG), gsrc) : nullptr;
    SlabPlan plg{0, 0, 0};
    if (GS) plg = slab_plan(gsrc, uint32_t(ne) * NP * 6u * uint32_t(sizeof(GT)));
    if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(bar, pl1.mid_bytes + pl2.mid_bytes + plg.mid_bytes);
        slab_issue(s1, src1, pl1, bar);
        if (CG) slab_issue(s2, src2, pl2, bar);
        if (GS) slab_issue(gdst, gsrc, plg, bar);
        // FP32: the factors read from global memory in phase 2 start towards L2
        // now (in FP64 a block computes so long that prefetched lines would be
        // evicted before phase 2 reads them)
        if (GM == kGLoad && sizeof(T) == 4) bulk_prefetch_l2(gsrc, uint32_t(ne) * NP * 6u * uint32_t(sizeof(GT)));
    }
    slab_edges(s1, src1, pl1, tid, nthreads);
    if (CG) slab_edges(s2, src2, pl2, tid, nthreads);
    if (GS) slab_edges(gdst, gsrc, plg, tid, nthreads);

    const int eb = tid / NQ2;
    const int ab = tid - eb * NQ2;
    const int a = ab % NQ, b = ab / NQ;
    const bool act = eb < ne;
    const int64_t nb = (e0 + eb) * NP;
    unsigned gw[PF ? NQ : 1][3];
    if (PF && act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const unsigned *gq = reinterpret_cast<const unsigned *>(G + 6 * (nb + k * NQ2 + b * NQ + a));
            gw[k][0] = __ldg(gq);
            gw[k][1] = __ldg(gq + 1);
            gw[k][2] = __ldg(gq + 2);
        }
    }
    const bool ok = mbar_wait_bounded(bar, phase, status);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, phase, nullptr);  // let copies in flight land before leaving
        return false;
    }

    const int rq = b * NQ2 + a * NQ;   // r line (j, k) = (a, b) of the slab: first node
    const int cq = b * NQ2 + a;        // s line (i, k) = (a, b) of the slab: first node, stride NQ
    const int tq = b * NQ + a;         // t line (i, j) = (a, b) of the slab: first node, stride NQ2
    const int rp = b * P2 + a * P1;    // the same lines in the padded U / V layout
    const int cp = b * P2 + a;
    const int tp = b * P1 + a;

    T xk[NQ];
    if (CG) {
        if (act) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const int q = eb * NP + k * NQ2 + tq;
                const T zq = PRE ? dinv[nb + k * NQ2 + tq] * s1[q] : s1[q];
                if (xs) xs[nb + k * NQ2 + tq] = fma(xalpha, s2[q], xs[nb + k * NQ2 + tq]);
                const T pn = fma(beta, s2[q], zq);
                s2[q] = pn;
                xk[k] = pn;
                p[nb + k * NQ2 + tq] = pn;
            }
        }
        __syncthreads();
    } else if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) xk[k] = s1[eb * NP + k * NQ2 + tq];
    }
    const T *SX = (CG ? s2 : s1) + eb * NP;
    T *SU = (CG ? regA : regB) + eb * NPP;
    T *SV = regC + eb * NPP;

    // ---- (1) gradient lines
    T ut[NQ];
    if (act) {
        T u[NQ], yl[NQ];
        if (ROT) {
            const int R = (ab / RPB) & (NQ - 1);
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = SX[rq + ((l + R) & (NQ - 1))];
            rotate_right<NQ, T>(u, R);
        } else {
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = SX[rq + l];
        }
        eo_apply<NQ, T>(u, yl, cd);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SU[rp + l] = yl[l];
        if (ROT) {
            const int R = b & (NQ - 1);
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = SX[cq + ((l + R) & (NQ - 1)) * NQ];
            rotate_right<NQ, T>(u, R);
        } else {
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = SX[cq + l * NQ];
        }
        eo_apply<NQ, T>(u, yl, cd);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SV[cp + l * P1] = yl[l];
        eo_apply<NQ, T>(xk, ut, cd);
    }
    __syncthreads();

    // ---- (2) geometric factors, node by node
    T wt[NQ];
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int pq = k * P2 + tp;
            const T ur = SU[pq], us = SV[pq];
            T g[6];
            if constexpr (PF) {
                const float2 g01 = bf16x2_to_float2(gw[k][0]), g23 = bf16x2_to_float2(gw[k][1]),
                             g45 = bf16x2_to_float2(gw[k][2]);
                g[0] = g01.x; g[1] = g01.y; g[2] = g23.x; g[3] = g23.y; g[4] = g45.x; g[5] = g45.y;
            } else if constexpr (GS) {
                load_g6_smem(reinterpret_cast<const GT *>(gdst) + 6 * (eb * NP + k * NQ2 + tq), g);
            } else {
                load_g6(G, nb + k * NQ2 + tq, g);
            }
            SU[pq] = g[0] * ur + g[1] * us + g[2] * ut[k];
            SV[pq] = g[1] * ur + g[3] * us + g[4] * ut[k];
            wt[k] = g[2] * ur + g[4] * us + g[5] * ut[k];
        }
    }
    __syncthreads();

    // ---- (3) divergence lines (in place: each line has one owner)
    T yt[NQ];
    if (act) {
        T u[NQ], yl[NQ];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SU[rp + l];
        eo_apply<NQ, T>(u, yl, ct);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SU[rp + l] = yl[l];
#pragma unroll
        for (int l = 0; l < NQ; ++l) u[l] = SV[cp + l * P1];
        eo_apply<NQ, T>(u, yl, ct);
#pragma unroll
        for (int l = 0; l < NQ; ++l) SV[cp + l * P1] = yl[l];
        eo_apply<NQ, T>(wt, yt, ct);
    }
    __syncthreads();

    // ---- (4) sum of the three directions
    T acc = T(0);
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int pq = k * P2 + tp;
            const T yv = (SU[pq] + SV[pq]) + yt[k];
            y[nb + k * NQ2 + tq] = yv;
            if (CG) acc = fma(SX[k * NQ2 + tq], yv, acc);
        }
    }
    if (CG) *part = acc;
    return true;
}

template <int NQ, typename T, typename GT, bool CG, bool PRE, int GM = kGLoad>
__global__ void __launch_bounds__(512) ax_lines_kernel(const AxLineArgs<T, GT> P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const AxArgs<T, GT> &A = P.a;
    if (CG && A.st->done) return;  // solve finished: the rest of the graph is a no-op

    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    T *regA = reinterpret_cast<T *>(smem + 16);
    const int64_t e0 = int64_t(blockIdx.x) * P.epb;
    const int ne = int(min(int64_t(P.epb), A.E - e0));
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    const T beta = CG ? T(A.st->beta) : T(0);
    // read before this launch's last block replaces it; only with a deferred x update
    const T xalpha = (CG && A.xs) ? T(A.st->alpha) : T(0);
    T part = T(0);
    if (!lines_group<NQ, T, GT, CG, PRE, GM>(A.x, A.y, A.p, A.G, P.d, P.dt, beta, xalpha, CG ? A.xs : nullptr,
                                             A.dinv, e0, ne, P.epb, regA, bar, 0u, A.status, &part))
        return;
    if (CG) {
        // the thread's partial is formed in T; the block sum in T for FP32
        // (FP64 for FP64), the grid sum in FP64 over groups of blocks (the
        // slab regions are free now and hold the block's partials)
        double bs;
        if constexpr (sizeof(T) == 4)
            bs = double(block_sum_f32(part, reinterpret_cast<float *>(regA)));
        else
            bs = block_sum_wide(double(part), reinterpret_cast<double *>(regA));
        if (publish_grouped(bs, A.partials, &A.st->ticket_ax)) {
            const double pap = finish_grouped(A.partials, &A.st->ticket_ax);
            if (threadIdx.x == 0) {
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
            if (sizeof(T) == 4) {
                c.eo[2 * (i * H + l)] = c.e[i * H + l];
                c.eo[2 * (i * H + l) + 1] = c.o[i * H + l];
            }
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

template <int NQ, typename T, typename GT, bool CG, bool PRE, int GM>
static int launch_lines_nq(const Problem *Pb, const AxLineArgs<T, GT> &L) {
    const int nt = line_threads(NQ, L.epb);
    if (L.epb < 1 || nt == 0) return set_error(SEM_EARG, "ax lines: elements per block out of range");
    const size_t sm = LineShape::smem(NQ, L.epb, int(sizeof(T)), GM == kGStaged ? 6 * int(sizeof(GT)) : 0);
    if (sm > size_t(227) * 1024) return set_error(SEM_EARG, "ax lines: shared memory per block too large");
    auto kern = ax_lines_kernel<NQ, T, GT, CG, PRE, GM>;
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
    if (CG && blocks > Pb->partials_cap) return set_error(SEM_ERANGE, "ax lines: more blocks than reduction slots");
    kern<<<unsigned(blocks), nt, sm, stream()>>>(L);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax_lines_kernel");
}

template <typename T, typename GT, bool CG, bool PRE = false, int GM = kGLoad>
static int launch_lines_any(const Problem *Pb, const AxLineArgs<T, GT> &L) {
    switch (Pb->nq) {
        case 2: return launch_lines_nq<2, T, GT, CG, PRE, GM>(Pb, L);
        case 3: return launch_lines_nq<3, T, GT, CG, PRE, GM>(Pb, L);
        case 4: return launch_lines_nq<4, T, GT, CG, PRE, GM>(Pb, L);
        case 5: return launch_lines_nq<5, T, GT, CG, PRE, GM>(Pb, L);
        case 6: return launch_lines_nq<6, T, GT, CG, PRE, GM>(Pb, L);
        case 7: return launch_lines_nq<7, T, GT, CG, PRE, GM>(Pb, L);
        case 8: return launch_lines_nq<8, T, GT, CG, PRE, GM>(Pb, L);
        case 9: return launch_lines_nq<9, T, GT, CG, PRE, GM>(Pb, L);
        case 10: return launch_lines_nq<10, T, GT, CG, PRE, GM>(Pb, L);
        default: return set_error(SEM_EARG, "ax lines: unsupported order");
    }
}

}  // namespace sem
