// sem_ax32p.cuh -- persistent, double-buffered FP32 local Poisson operator
// for the HBM-bound inner solves of mixed-precision refinement.
//
// Same arithmetic as ax_kernel<.., float, GT, ..> (sem_ax_kernel.cuh), but a
// fixed grid of CTAs walks the element groups, and each CTA keeps two stages
// of shared memory: while it computes group t from stage t%2, the TMA engine
// is already filling the other stage with group t+grid's slabs -- the input
// vector(s) and the group's geometric factors (stored interleaved per node,
// 12 bytes in BF16 or 24 in FP32) -- so HBM always has a stage of bytes in
// flight per CTA.  Each stage has its own mbarrier; the k-th use of stage s
// completes phase k mod 2.  Before a stage is refilled, the CTA has finished
// with it (block barrier) and a proxy fence orders the threads' earlier
// shared-memory writes before the engine's.
//
// CG mode: stage A holds r, stage B holds p; p = r + beta p is written back
// into B and to global memory; the r-direction products go into A (free once
// p is formed).  Plain mode: A holds x; B takes the r-direction products.
#pragma once

#include "sem_ax_kernel.cuh"

namespace sem {

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <int NQ, int EPB, typename GT>
struct AxpShape {
    static constexpr int NQ2 = NQ * NQ;
    static constexpr int NP = NQ2 * NQ;
    static constexpr int NTA = NQ2 * EPB;
    static constexpr int NT = (NTA + 31) / 32 * 32;
    static constexpr int SLAB = (EPB * NP + 8 + 3) / 4 * 4;                      // floats, + 16 B slack
    static constexpr int GBYTES = (EPB * NP * 6 * int(sizeof(GT)) + 32 + 15) / 16 * 16;
    static constexpr int STAGE = 2 * SLAB * 4 + GBYTES;                          // bytes per stage
    static constexpr size_t SMEM = 32 + 2 * size_t(STAGE) + size_t(SLAB) * 4;
};

// Elements per group: ~256 threads; FP32 factors take twice the bytes, so
// fewer elements per stage.
template <int NQ, typename GT>
struct AxpEpb {
    static constexpr int bf16 = NQ <= 2 ? 64 : NQ == 3 ? 28 : NQ == 4 ? 16 : NQ == 5 ? 10
                              : NQ == 6 ? 7 : NQ == 7 ? 5 : NQ == 8 ? 4 : NQ == 9 ? 3 : 2;
    static constexpr int f32 = NQ <= 2 ? 32 : NQ == 3 ? 14 : NQ == 4 ? 8 : NQ == 5 ? 5
                             : NQ == 6 ? 3 : NQ <= 8 ? 2 : NQ == 9 ? 1 : 1;
    static constexpr int value = sizeof(GT) == 2 ? bf16 : f32;
};

template <int NQ, int EPB, typename GT, bool CG>
__global__ void __launch_bounds__(AxpShape<NQ, EPB, GT>::NT)
ax32p_kernel(const AxArgs<float, GT> P, int ngroups) {
    using S = AxpShape<NQ, EPB, GT>;
    constexpr int NQ2 = S::NQ2, NP = S::NP;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[32];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);     // bar[0], bar[1]
    unsigned char *stages = smem + 32;
    float *ws_buf = reinterpret_cast<float *>(stages + 2 * S::STAGE);

    if (CG && P.st->done) return;  // solve finished: the rest of the graph is a no-op

    const int tid = threadIdx.x;
    const int eb = tid / NQ2;
    const int ij = tid - eb * NQ2;
    const int i = ij % NQ, j = ij / NQ;

    auto stA = [&](int s) { return reinterpret_cast<float *>(stages + s * S::STAGE); };
    auto stB = [&](int s) { return reinterpret_cast<float *>(stages + s * S::STAGE) + S::SLAB; };
    auto stG = [&](int s) { return stages + s * S::STAGE + 2 * S::SLAB * 4; };
    auto group_ne = [&](int g) { return int(min(int64_t(EPB), P.E - int64_t(g) * EPB)); };
    auto srcA = [&](int g) { return P.x + int64_t(g) * EPB * NP; };
    auto srcB = [&](int g) { return P.p + int64_t(g) * EPB * NP; };
    auto srcG = [&](int g) {
        return reinterpret_cast<const unsigned char *>(P.G) + int64_t(g) * EPB * NP * 6 * int64_t(sizeof(GT));
    };
    // TMA part of a group's copies into stage s (thread 0 only)
    auto issue = [&](int g, int s) {
        const int ne = group_ne(g);
        const uint32_t vb = uint32_t(ne) * NP * 4u, gb = uint32_t(ne) * NP * 6u * uint32_t(sizeof(GT));
        const SlabPlan pa = slab_plan(srcA(g), vb);
        const SlabPlan pb = CG ? slab_plan(srcB(g), vb) : SlabPlan{0, 0, 0};
        const SlabPlan pg = slab_plan(srcG(g), gb);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar[s], pa.mid_bytes + pb.mid_bytes + pg.mid_bytes);
        slab_issue(slab_dst(stA(s), srcA(g)), srcA(g), pa, &bar[s]);
        if (CG) slab_issue(slab_dst(stB(s), srcB(g)), srcB(g), pb, &bar[s]);
        slab_issue(slab_dst(stG(s), srcG(g)), srcG(g), pg, &bar[s]);
    };

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    __syncthreads();
    int g = blockIdx.x;
    if (tid == 0 && g < ngroups) issue(g, 0);

    double acc_total = 0.0;
    for (int t = 0; g < ngroups; ++t, g += gridDim.x) {
        const int s = t & 1;
        const uint32_t parity = uint32_t(t >> 1) & 1u;
        const int gn = g + gridDim.x;
        if (tid == 0 && gn < ngroups) issue(gn, s ^ 1);
        const bool ok = mbar_wait_bounded(&bar[s], parity, P.status);
        if (__syncthreads_or(!ok)) {
            // drain this stage and the one just issued before leaving
            mbar_wait_bounded(&bar[s], parity, nullptr);
            if (gn < ngroups) mbar_wait_bounded(&bar[s ^ 1], uint32_t((t + 1) >> 1) & 1u, nullptr);
            return;
        }
        const int ne = group_ne(g);
        const uint32_t vb = uint32_t(ne) * NP * 4u, gb = uint32_t(ne) * NP * 6u * uint32_t(sizeof(GT));
        float *sa = slab_dst(stA(s), srcA(g));
        float *sb = CG ? slab_dst(stB(s), srcB(g)) : nullptr;
        const GT *sg = reinterpret_cast<const GT *>(slab_dst(stG(s), srcG(g)));
        slab_edges(sa, srcA(g), slab_plan(srcA(g), vb), tid, S::NT);
        if (CG) slab_edges(sb, srcB(g), slab_plan(srcB(g), vb), tid, S::NT);
        slab_edges(reinterpret_cast<unsigned char *>(const_cast<GT *>(sg)), srcG(g), slab_plan(srcG(g), gb), tid,
                   S::NT);
        __syncthreads();

        const bool act = (tid < S::NTA) && (eb < ne);
        const int64_t nb = (int64_t(g) * EPB + eb) * NP;
        float xk[NQ];
        if (CG) {
            const float beta = float(P.st->beta);
            if (act) {
#pragma unroll
                for (int k = 0; k < NQ; ++k) {
                    const int q = eb * NP + k * NQ2 + ij;
                    const float pn = fmaf(beta, sb[q], sa[q]);
                    sb[q] = pn;
                    xk[k] = pn;
                    P.p[nb + k * NQ2 + ij] = pn;
                }
            }
            __syncthreads();
        } else if (act) {
#pragma unroll
            for (int k = 0; k < NQ; ++k) xk[k] = sa[eb * NP + k * NQ2 + ij];
        }
        const float *sx = (CG ? sb : sa) + eb * NP;
        float *s_wr = (CG ? stA(s) : stB(s)) + eb * NP;
        float *s_ws = ws_buf + eb * NP;

        float wt[NQ];
        if (act) {
            float Di[NQ], Dj[NQ];
#pragma unroll
            for (int l = 0; l < NQ; ++l) {
                Di[l] = P.D[i * NQ + l];
                Dj[l] = P.D[j * NQ + l];
            }
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                float ur = 0.f, us = 0.f, ut = 0.f;
#pragma unroll
                for (int l = 0; l < NQ; ++l) {
                    ur = fmaf(Di[l], sx[k * NQ2 + j * NQ + l], ur);
                    us = fmaf(Dj[l], sx[k * NQ2 + l * NQ + i], us);
                    ut = fmaf(P.D[k * NQ + l], xk[l], ut);
                }
                float gv[6];
                load_g6_smem(sg + 6 * (eb * NP + k * NQ2 + ij), gv);
                s_wr[k * NQ2 + ij] = gv[0] * ur + gv[1] * us + gv[2] * ut;
                s_ws[k * NQ2 + ij] = gv[1] * ur + gv[3] * us + gv[4] * ut;
                wt[k] = gv[2] * ur + gv[4] * us + gv[5] * ut;
            }
        }
        __syncthreads();
        if (act) {
            float Dti[NQ], Dtj[NQ];
#pragma unroll
            for (int l = 0; l < NQ; ++l) {
                Dti[l] = P.D[l * NQ + i];
                Dtj[l] = P.D[l * NQ + j];
            }
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                float yv = 0.f;
#pragma unroll
                for (int l = 0; l < NQ; ++l) yv = fmaf(Dti[l], s_wr[k * NQ2 + j * NQ + l], yv);
#pragma unroll
                for (int l = 0; l < NQ; ++l) yv = fmaf(Dtj[l], s_ws[k * NQ2 + l * NQ + i], yv);
#pragma unroll
                for (int l = 0; l < NQ; ++l) yv = fmaf(P.D[l * NQ + k], wt[l], yv);
                P.y[nb + k * NQ2 + ij] = yv;
                if (CG) acc = fmaf(xk[k], yv, acc);
            }
            if (CG) acc_total += double(acc);
        }
        // stage s and ws_buf are free for the next refill: order this thread's
        // shared-memory writes before the TMA engine's, then meet
        fence_proxy_async_smem();
        __syncthreads();
    }
    if (CG) {
        const double bs = block_sum(acc_total, red);
        if (publish_partial(bs, P.partials, &P.st->ticket_ax)) {
            const double pap = finish_partials(P.partials, int(gridDim.x), &P.st->ticket_ax, red);
            if (tid == 0) {
                P.st->pap = pap;
                P.st->alpha = P.st->rho / pap;
            }
        }
    }
}

}  // namespace sem
