// sem_ax32.cu -- FP32 instantiations of the local Poisson operator for the
// inner solves of mixed-precision iterative refinement: FP32 vectors and
// arithmetic, geometric factors stored in FP32 (24 B/node) or BF16
// (12 B/node) and widened exactly to FP32 on load; the CG variant's <p, A p>
// is reduced across threads and blocks in FP64.  Also the one-time
// conversion of the FP64 geometric factors (round to nearest even).
#include <cuda_bf16.h>

#include "sem_ax_kernel.cuh"

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

int prepare_ax32(const Problem *Pb) {
    const int rc = prepare_ax_any<float, float>(Pb);
    return rc != SEM_OK ? rc : prepare_ax_any<float, __nv_bfloat16>(Pb);
}

int launch_ax32(const Problem *Pb, const float *x, float *y, int gprec) {
    if (gprec == kGF32) {
        AxArgs<float, float> a = ax_args<float, float>(Pb, static_cast<const float *>(Pb->G32), Pb->partials, Pb->st_in);
        a.x = x;
        a.y = y;
        return launch_ax_any<float, float, false>(Pb, a);
    }
    AxArgs<float, __nv_bfloat16> a =
        ax_args<float, __nv_bfloat16>(Pb, static_cast<const __nv_bfloat16 *>(Pb->G16), Pb->partials, Pb->st_in);
    a.x = x;
    a.y = y;
    return launch_ax_any<float, __nv_bfloat16, false>(Pb, a);
}

int launch_ax32_cg(const Problem *Pb, int gprec) {
    if (gprec == kGF32) {
        AxArgs<float, float> a = ax_args<float, float>(Pb, static_cast<const float *>(Pb->G32), Pb->partials, Pb->st_in);
        a.x = Pb->r32;
        a.y = Pb->w32;
        a.p = Pb->p32;
        return launch_ax_any<float, float, true>(Pb, a);
    }
    AxArgs<float, __nv_bfloat16> a =
        ax_args<float, __nv_bfloat16>(Pb, static_cast<const __nv_bfloat16 *>(Pb->G16), Pb->partials, Pb->st_in);
    a.x = Pb->r32;
    a.y = Pb->w32;
    a.p = Pb->p32;
    return launch_ax_any<float, __nv_bfloat16, true>(Pb, a);
}

}  // namespace sem
