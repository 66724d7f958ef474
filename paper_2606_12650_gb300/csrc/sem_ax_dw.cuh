// sem_ax_dw.cuh -- the FP64 local Poisson operator evaluated in double-word
// FP32 arithmetic (pairs of FP32 numbers) on the FP32 pipe.
//
// Same map, thread roles and phases as the line kernel (sem_ax_lines.cuh):
// whole r/s/t lines per thread, the even-odd split of D and D^T, the element
// slab staged by the TMA engine.  Inputs and outputs stay FP64 in HBM (x or
// r, p; y or w; the CG recurrences and reductions are untouched).  Inside the
// kernel every value is a double-word number v = h + l of two FP32 numbers:
//   - the derivative sweeps, the geometric-factor product and the sum of the
//     three directions use error-free transformations -- Knuth's TwoSum
//     (TAOCP vol. 2, 4.2.2, Thm B) for sums of the high parts, Dekker's
//     product (1971) formed with one FMA for products of the high parts --
//     and FP32 arithmetic for the low-order terms, which are ~2^-24 of the
//     value (the "Dot2" accumulation of Ogita, Rump and Oishi, SISC 2005,
//     extended to double-word operands); l is not renormalised after each
//     operation (the high part keeps the leading 24 bits; cancellation moves
//     no error above 2^-48 of the operands' size);
//   - the constants (even-odd halves of D, D^T) and the geometric factors are
//     rounded to double-word once (h = rn(d), l = rn(d - h)), the factors by
//     set-up into a [nL][6] (h, l) array of the same 48 bytes per node as FP64.
// Each value carries ~48 significant bits: the operator matches the FP64
// direct evaluation to ~2e-14 of max|y| on random input (FP64: ~6e-16), well
// inside the 1e-13 parity bar, for inputs whose magnitudes lie within FP32's
// exponent range with room for the low part (~[2^-100, 2^126]: below it the
// low parts become subnormal and precision falls towards FP32's).
// Why: GB300 executes FP64 at 1/64 of its FP32 rate, and the FP64 line kernel is bound by its
// ~50 DFMA per node; here a node costs ~450 FP32 operations (~7 DFMA worth),
// which moves the bound from the FP64 pipe towards HBM bandwidth.
#pragma once

#include "sem_ax_lines.cuh"
#include "sem_dw.cuh"

namespace sem {

// Even-odd coefficients of a centro-antisymmetric matrix (as EoMat) in
// double-word form.
struct EoMatDW {
    dwf e[25];
    dwf o[30];
    dwf m[5];
};

// y = M u by the even-odd split (the same sums as eo_apply), double-word.
template <int NQ>
__device__ __forceinline__ void eo_apply_dw(const dwf (&u)[NQ], dwf (&y)[NQ], const EoMatDW &c) {
    constexpr int H = NQ / 2;
    constexpr bool ODD = (NQ & 1) != 0;
    dwf ue[H], uo[H];
#pragma unroll
    for (int l = 0; l < H; ++l) {
        ue[l] = dw_add(u[l], u[NQ - 1 - l]);
        uo[l] = dw_sub(u[l], u[NQ - 1 - l]);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        dwf a = dw_mul(c.e[i * H], ue[0]);
        dwf b = dw_mul(c.o[i * H], uo[0]);
#pragma unroll
        for (int l = 1; l < H; ++l) {
            a = dw_fma(c.e[i * H + l], ue[l], a);
            b = dw_fma(c.o[i * H + l], uo[l], b);
        }
        if (ODD) a = dw_fma(c.m[i], u[H], a);
        y[i] = dw_add(a, b);
        y[NQ - 1 - i] = dw_sub(b, a);
    }
    if (ODD) {
        dwf b = dw_mul(c.o[H * H], uo[0]);
#pragma unroll
        for (int l = 1; l < H; ++l) b = dw_fma(c.o[H * H + l], uo[l], b);
        y[H] = b;
    }
}

// Host: even-odd halves of M (row-major nq x nq), formed in FP64, then split
// into double-word pairs (h = rn(d), l = rn(d - h)).
inline dwf dw_split_host(double d) {
    const float h = float(d);
    return {h, float(d - double(h))};
}

inline EoMatDW eo_coefficients_dw(const double *M, int nq) {
    EoMatDW c{};
    const int N = nq - 1, H = nq / 2;
    for (int i = 0; i < H; ++i)
        for (int l = 0; l < H; ++l) {
            c.e[i * H + l] = dw_split_host(0.5 * (M[i * nq + l] + M[i * nq + N - l]));
            c.o[i * H + l] = dw_split_host(0.5 * (M[i * nq + l] - M[i * nq + N - l]));
        }
    if (nq & 1) {
        for (int l = 0; l < H; ++l) c.o[H * H + l] = dw_split_host(0.5 * (M[H * nq + l] - M[H * nq + N - l]));
        for (int i = 0; i < H; ++i) c.m[i] = dw_split_host(M[i * nq + H]);
    }
    return c;
}

struct AxDwArgs {
    AxArgs<double, double> a;   // FP64 vectors, state, partials (a.G unused)
    const float *Gdw;           // [nL][6][2]: (h, l) of each FP64 factor
    EoMatDW d;                  // of D   (gradient)
    EoMatDW dt;                 // of D^T (divergence)
    int epb;                    // elements per block
};

// The six double-word factors of one node: three 16-byte loads.
__device__ __forceinline__ void load_g6_dw(const float *Gdw, int64_t node, dwf (&g)[6]) {
    const float4 *q = reinterpret_cast<const float4 *>(Gdw + 12 * node);
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    g[0] = {a.x, a.y}; g[1] = {a.z, a.w}; g[2] = {b.x, b.y};
    g[3] = {b.z, b.w}; g[4] = {c.x, c.y}; g[5] = {c.z, c.w};
}

// One group of ne (<= epb) elements starting at element e0 (the line
// kernel's lines_group, double-word).  regA: 16-byte aligned shared memory of
// 3 LineShape::region(N+1, epb, 8) doubles; the FP64 slab is staged there
// and converted in place to double-word values (same 8 bytes per node); U and
// V hold double-word values in the padded layout.  CG mode: xs += xalpha
// p_old and p = r + beta p (PRE: M^-1 r + beta p) in FP64, p written back in
// FP64; *part receives this thread's <p, A_local p> partial.  Returns false
// if the slab copy timed out (status set, copies drained).
template <int NQ, bool CG, bool PRE>
__device__ __forceinline__ bool lines_group_dw(const double *x, double *y, double *p, const float *Gdw,
                                               const EoMatDW &cd, const EoMatDW &ct, double beta, double xalpha,
                                               double *xs, const double *dinv, int64_t e0, int ne, int epb,
                                               double *regA, uint64_t *bar, uint32_t phase, int32_t *status,
                                               double *part) {
    constexpr int NQ2 = NQ * NQ, NP = NQ2 * NQ;
    constexpr int P1 = LinePad<NQ>::P1, P2 = LinePad<NQ>::P2, NPP = LinePad<NQ>::NPP;
    // N+1 = 8: rows of 8 values 8 bytes wide start 64 B apart, two to a
    // 128-byte bank row: rotated reads as in the FP64 line kernel
    constexpr bool ROT = NQ == 8;
    constexpr int RPB = 2;
    const int RG = LineShape::region(NQ, epb, int(sizeof(double)));
    double *regB = regA + RG;
    double *regC = regB + RG;
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;

    // ---- (0) stage the FP64 slab(s): TMA for the aligned middle, plain loads for the edges
    const uint32_t bytes = uint32_t(ne) * NP * uint32_t(sizeof(double));
    const double *src1 = x + e0 * NP;                 // x (plain) or r (CG)
    const double *src2 = CG ? p + e0 * NP : nullptr;  // p (CG)
    double *s1 = slab_dst(regA, src1);
    double *s2 = CG ? slab_dst(regB, src2) : nullptr;
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

    const int eb = tid / NQ2;
    const int ab = tid - eb * NQ2;
    const int a = ab % NQ, b = ab / NQ;
    const bool act = eb < ne;
    const int64_t nb = (e0 + eb) * NP;
    // CG: the x values of the thread's t line (deferred update) are loaded
    // before the slab wait, so their latency overlaps the copy
    double xpre[CG ? NQ : 1];
    if (CG && act && xs) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) xpre[k] = xs[nb + k * NQ2 + b * NQ + a];
    }
    const bool ok = mbar_wait_bounded(bar, phase, status);
    if (__syncthreads_or(!ok)) {
        mbar_wait_bounded(bar, phase, nullptr);  // let copies in flight land before leaving
        return false;
    }

    const int rq = b * NQ2 + a * NQ;   // r line (j, k) = (a, b) of the slab: first node
    const int cq = b * NQ2 + a;        // s line (i, k) = (a, b): first node, stride NQ
    const int tq = b * NQ + a;         // t line (i, j) = (a, b): first node, stride NQ2
    const int rp = b * P2 + a * P1;    // the same lines in the padded U / V layout
    const int cp = b * P2 + a;
    const int tp = b * P1 + a;

    // ---- (0b) the thread's t line: CG prologue in FP64, then to double-word
    // in place (each node is converted by the one thread that owns its t line;
    // the converted slab is read again for <p, y> in phase 4)
    dwf xk[NQ];
    double *slab = CG ? s2 : s1;
    dwf *SXw = reinterpret_cast<dwf *>(slab);
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int q = eb * NP + k * NQ2 + tq;
            double v;
            if (CG) {
                const double zq = PRE ? dinv[nb + k * NQ2 + tq] * s1[q] : s1[q];
                if (xs) xs[nb + k * NQ2 + tq] = fma(xalpha, s2[q], xpre[k]);
                v = fma(beta, s2[q], zq);
                p[nb + k * NQ2 + tq] = v;
            } else {
                v = s1[q];
            }
            xk[k] = dw_from_double(v);
            SXw[q] = xk[k];
        }
    }
    __syncthreads();
    const dwf *SX = SXw + eb * NP;
    dwf *SU = reinterpret_cast<dwf *>(CG ? regA : regB) + eb * NPP;
    dwf *SV = reinterpret_cast<dwf *>(regC) + eb * NPP;

    // ---- (1) gradient lines.  FOLD: the r and s lines share one copy of the
    // (long, fully unrolled) double-word contraction -- a two-pass loop over
    // (first node, stride, rotation, destination) -- since the unrolled body
    // outgrows the instruction cache (no-instruction stalls; N+1 = 8:
    // 373 -> 358 us).  Not at N+1 = 9, where the loop's addressing takes 92
    // registers instead of 64.
    constexpr bool FOLD = NQ != 9;
    dwf ut[NQ];
    if (act) {
        dwf u[NQ], yl[NQ];
        auto rs_line = [&](int d) {
            const int q0 = d ? cq : rq, st = d ? NQ : 1;
            const int R = ROT ? (d ? (b & (NQ - 1)) : ((ab / RPB) & (NQ - 1))) : 0;
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = SX[q0 + (ROT ? ((l + R) & (NQ - 1)) : l) * st];
            if (ROT) rotate_right<NQ, dwf>(u, R);
            eo_apply_dw<NQ>(u, yl, cd);
            dwf *dst = d ? SV + cp : SU + rp;
            const int ds = d ? P1 : 1;
#pragma unroll
            for (int l = 0; l < NQ; ++l) dst[l * ds] = yl[l];
        };
        if constexpr (FOLD) {
#pragma unroll 1
            for (int d = 0; d < 2; ++d) rs_line(d);
        } else {
            rs_line(0);
            rs_line(1);
        }
        eo_apply_dw<NQ>(xk, ut, cd);   // the t line, from the registers of the prologue
    }
    __syncthreads();

    // ---- (2) geometric factors, node by node
    dwf wt[NQ];
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int pq = k * P2 + tp;
            const dwf ur = SU[pq], us = SV[pq];
            dwf g[6];
            load_g6_dw(Gdw, nb + k * NQ2 + tq, g);
            SU[pq] = dw_fma(g[2], ut[k], dw_fma(g[1], us, dw_mul(g[0], ur)));
            SV[pq] = dw_fma(g[4], ut[k], dw_fma(g[3], us, dw_mul(g[1], ur)));
            wt[k] = dw_fma(g[5], ut[k], dw_fma(g[4], us, dw_mul(g[2], ur)));
        }
    }
    __syncthreads();

    // ---- (3) divergence lines (in place: each line has one owner); FOLD as
    // in phase 1
    dwf yt[NQ];
    if (act) {
        dwf u[NQ], yl[NQ];
        auto rs_line = [&](int d) {
            dwf *line = d ? SV + cp : SU + rp;
            const int ls = d ? P1 : 1;
#pragma unroll
            for (int l = 0; l < NQ; ++l) u[l] = line[l * ls];
            eo_apply_dw<NQ>(u, yl, ct);
#pragma unroll
            for (int l = 0; l < NQ; ++l) line[l * ls] = yl[l];
        };
        if constexpr (FOLD) {
#pragma unroll 1
            for (int d = 0; d < 2; ++d) rs_line(d);
        } else {
            rs_line(0);
            rs_line(1);
        }
        eo_apply_dw<NQ>(wt, yt, ct);   // the t line (registers), out of the loop, whose
                                       // iterations would otherwise hold wt and yt live together
    }
    __syncthreads();

    // ---- (4) sum of the three directions, back to FP64; <p, y> in double-word
    dwf acc = {0.f, 0.f};
    if (act) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const int pq = k * P2 + tp;
            const dwf yv = dw_add(dw_add(SU[pq], SV[pq]), yt[k]);
            y[nb + k * NQ2 + tq] = dw_to_double(yv);
            if (CG) acc = dw_fma(SX[k * NQ2 + tq], yv, acc);
        }
    }
    if (CG) *part = dw_to_double(acc);
    return true;
}

template <int NQ, bool CG, bool PRE>
__global__ void __launch_bounds__(512) ax_dw_kernel(const AxDwArgs P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const AxArgs<double, double> &A = P.a;
    if (CG && A.st->done) return;  // solve finished: the rest of the graph is a no-op

    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    double *regA = reinterpret_cast<double *>(smem + 16);
    const int64_t e0 = int64_t(blockIdx.x) * P.epb;
    const int ne = int(min(int64_t(P.epb), A.E - e0));
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    const double beta = CG ? A.st->beta : 0.0;
    // read before this launch's last block replaces it; only with a deferred x update
    const double xalpha = (CG && A.xs) ? A.st->alpha : 0.0;
    double part = 0.0;
    if (!lines_group_dw<NQ, CG, PRE>(A.x, A.y, A.p, P.Gdw, P.d, P.dt, beta, xalpha, CG ? A.xs : nullptr, A.dinv,
                                     e0, ne, P.epb, regA, bar, 0u, A.status, &part))
        return;
    if (CG) {
        const double bs = block_sum_wide(part, regA);
        if (publish_grouped(bs, A.partials, &A.st->ticket_ax)) {
            const double pap = finish_grouped(A.partials, &A.st->ticket_ax);
            if (threadIdx.x == 0) {
                A.st->pap = pap;
                A.st->alpha = A.st->rho / pap;
            }
        }
    }
}

}  // namespace sem
