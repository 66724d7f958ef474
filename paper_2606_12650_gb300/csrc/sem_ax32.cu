// sem_ax32.cu -- the FP32 local Poisson operator for the inner solves of
// mixed-precision iterative refinement (persistent, double-buffered kernel
// of sem_ax32p.cuh): FP32 vectors and arithmetic, geometric factors stored in
// FP32 (24 B/node) or BF16 (12 B/node) and widened exactly to FP32; the CG
// variant's <p, A p> is reduced across threads and blocks in FP64.  Also the
// one-time conversion of the FP64 geometric factors (round to nearest even).
#include <cuda_bf16.h>

#include <algorithm>

#include "sem_ax32p.cuh"

namespace sem {

__global__ void g_to_f32_kernel(const double *__restrict__ G, float *__restrict__ out, int64_t n) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n) out[t] = __double2float_rn(G[t]);
}

// FP64 -> BF16 with one round-to-nearest-even step on the FP64 bit pattern
// (8 significant bits kept, ties to even; below the BF16 normal range -> 0).
__device__ __forceinline__ unsigned short f64_to_bf16_rne(double x) {
    const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned sign = unsigned(u >> 63);
    int ex = int((u >> 52) & 0x7ff);
    const unsigned long long man = u & ((1ull << 52) - 1);
    if (ex == 0x7ff) return (unsigned short)((sign << 15) | 0x7f80u | (man ? 0x40u : 0u));  // inf / nan
    unsigned long long keep = man >> 45;
    const unsigned long long rem = man & ((1ull << 45) - 1), half = 1ull << 44;
    if (rem > half || (rem == half && (keep & 1ull))) ++keep;
    if (keep == 128ull) {
        keep = 0;
        ++ex;
    }
    const int eb = ex - 1023 + 127;
    if (ex == 0 || eb <= 0) return (unsigned short)(sign << 15);
    if (eb >= 255) return (unsigned short)((sign << 15) | 0x7f80u);
    return (unsigned short)((sign << 15) | (unsigned(eb) << 7) | unsigned(keep));
}

__global__ void g_to_bf16_kernel(const double *__restrict__ G, unsigned short *__restrict__ out, int64_t n) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n) out[t] = f64_to_bf16_rne(G[t]);
}

int convert_geometry(const Problem *Pb, int gprec, void *out) {
    const int64_t n = 6 * Pb->nL;
    const unsigned blocks = unsigned((n + 255) / 256);
    if (gprec == kGF32)
        g_to_f32_kernel<<<blocks, 256, 0, stream()>>>(Pb->G, static_cast<float *>(out), n);
    else
        g_to_bf16_kernel<<<blocks, 256, 0, stream()>>>(Pb->G, static_cast<unsigned short *>(out), n);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "geometry conversion");
}

// Persistent launch: as many CTAs as fit on the GPU at once, each walking
// element groups with a two-stage TMA pipeline (sem_ax32p.cuh).
template <int NQ, typename GT, bool CG>
static int ax32p_setup(int *per_sm) {
    constexpr int EPB = AxpEpb<NQ, GT>::value;
    using S = AxpShape<NQ, EPB, GT>;
    static int occ = 0;
    if (!occ) {
        auto kern = ax32p_kernel<NQ, EPB, GT, CG>;
        int rc = cuda_check(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(S::SMEM)),
                            "ax32p: smem attribute");
        if (rc != SEM_OK) return rc;
        int o = 0;
        rc = cuda_check(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, S::NT, S::SMEM), "ax32p: occupancy");
        if (rc != SEM_OK) return rc;
        if (o < 1) return set_error(SEM_ECUDA, "ax32p: kernel does not fit on an SM");
        occ = o;
    }
    *per_sm = occ;
    return SEM_OK;
}

template <int NQ, typename GT, bool CG>
static int launch_ax32p_nq(const Problem *Pb, const AxArgs<float, GT> &a) {
    constexpr int EPB = AxpEpb<NQ, GT>::value;
    using S = AxpShape<NQ, EPB, GT>;
    int per_sm = 0;
    const int rc = ax32p_setup<NQ, GT, CG>(&per_sm);
    if (rc != SEM_OK) return rc;
    const int64_t ngroups = (Pb->E + EPB - 1) / EPB;
    const int64_t blocks = std::min<int64_t>(ngroups, int64_t(sm_count()) * per_sm);
    ax32p_kernel<NQ, EPB, GT, CG><<<unsigned(blocks), S::NT, S::SMEM, stream()>>>(a, int(ngroups));
    count_launches(1);
    return cuda_check(cudaGetLastError(), "ax32p_kernel");
}

template <typename GT, bool CG>
static int launch_ax32p(const Problem *Pb, const AxArgs<float, GT> &a) {
    switch (Pb->nq) {
        case 2: return launch_ax32p_nq<2, GT, CG>(Pb, a);
        case 3: return launch_ax32p_nq<3, GT, CG>(Pb, a);
        case 4: return launch_ax32p_nq<4, GT, CG>(Pb, a);
        case 5: return launch_ax32p_nq<5, GT, CG>(Pb, a);
        case 6: return launch_ax32p_nq<6, GT, CG>(Pb, a);
        case 7: return launch_ax32p_nq<7, GT, CG>(Pb, a);
        case 8: return launch_ax32p_nq<8, GT, CG>(Pb, a);
        case 9: return launch_ax32p_nq<9, GT, CG>(Pb, a);
        case 10: return launch_ax32p_nq<10, GT, CG>(Pb, a);
        default: return set_error(SEM_EARG, "ax32: unsupported order");
    }
}

template <typename GT>
static int prepare_gt(int nq) {
    int per_sm = 0, rc = SEM_OK;
    switch (nq) {
#define SEM_PREP32(Q)                                                   \
    case Q:                                                             \
        rc = ax32p_setup<Q, GT, false>(&per_sm);                        \
        return rc != SEM_OK ? rc : ax32p_setup<Q, GT, true>(&per_sm);
        SEM_PREP32(2) SEM_PREP32(3) SEM_PREP32(4) SEM_PREP32(5) SEM_PREP32(6)
        SEM_PREP32(7) SEM_PREP32(8) SEM_PREP32(9) SEM_PREP32(10)
#undef SEM_PREP32
        default: return set_error(SEM_EARG, "ax32: unsupported order");
    }
}

int prepare_ax32(const Problem *Pb) {
    const int rc = prepare_gt<float>(Pb->nq);
    return rc != SEM_OK ? rc : prepare_gt<__nv_bfloat16>(Pb->nq);
}

int launch_ax32(const Problem *Pb, const float *x, float *y, int gprec) {
    const TuneChoice c = tune_get(tune_kind_of_gprec(gprec), Pb->nq);
    if (c.variant == kAxLines || c.variant == kAxLinesPrefetch || c.variant == kAxLinesStaged)
        return launch_lines32(Pb, x, y, gprec, false, c.epb,
                              c.variant == kAxLinesPrefetch ? 1 : (c.variant == kAxLinesStaged ? 2 : 0));
    if (gprec == kGF32) {
        AxArgs<float, float> a = ax_args<float, float>(Pb, static_cast<const float *>(Pb->G32), Pb->partials, Pb->st_in);
        a.x = x;
        a.y = y;
        return launch_ax32p<float, false>(Pb, a);
    }
    AxArgs<float, __nv_bfloat16> a =
        ax_args<float, __nv_bfloat16>(Pb, static_cast<const __nv_bfloat16 *>(Pb->G16), Pb->partials, Pb->st_in);
    a.x = x;
    a.y = y;
    return launch_ax32p<__nv_bfloat16, false>(Pb, a);
}

int launch_ax32_cg(const Problem *Pb, int gprec) {
    const TuneChoice c = tune_get(tune_kind_of_gprec(gprec), Pb->nq);
    if (c.variant == kAxLines || c.variant == kAxLinesPrefetch || c.variant == kAxLinesStaged)
        return launch_lines32(Pb, nullptr, nullptr, gprec, true, c.epb,
                              c.variant == kAxLinesPrefetch ? 1 : (c.variant == kAxLinesStaged ? 2 : 0));
    if (gprec == kGF32) {
        AxArgs<float, float> a = ax_args<float, float>(Pb, static_cast<const float *>(Pb->G32), Pb->partials, Pb->st_in);
        a.x = Pb->r32;
        a.y = Pb->w32;
        a.p = Pb->p32;
        return launch_ax32p<float, true>(Pb, a);
    }
    AxArgs<float, __nv_bfloat16> a =
        ax_args<float, __nv_bfloat16>(Pb, static_cast<const __nv_bfloat16 *>(Pb->G16), Pb->partials, Pb->st_in);
    a.x = Pb->r32;
    a.y = Pb->w32;
    a.p = Pb->p32;
    return launch_ax32p<__nv_bfloat16, true>(Pb, a);
}

}  // namespace sem
