// sem_ax_lines32.cu -- FP32 instantiations of the line kernel
// (sem_ax_lines.cuh) for the inner solves of mixed-precision refinement:
// geometric factors stored in FP32 or BF16, plain and CG operator.
#include <cuda_bf16.h>

#include "sem_ax_lines.cuh"

namespace sem {

int launch_lines32(const Problem *P, const float *x, float *y, int gprec, bool cg, int epb, int gm) {
    const int gb = gprec == kGF32 ? 24 : 12;
    if (!lines_epb_ok(P->nq, epb, sizeof(float), gm == kGStaged ? gb : 0))
        return set_error(SEM_EARG, "ax lines: bad elements per block");
    if (gprec == kGF32) {
        AxArgs<float, float> a = ax_args<float, float>(P, static_cast<const float *>(P->G32), P->partials, P->st_in);
        if (cg) {
            a.x = P->r32;
            a.y = P->w32;
            a.p = P->p32;
            if (gm == kGStaged)
                return launch_lines_any<float, float, true, false, kGStaged>(P, line_args(a, P->oc.D, P->nq, epb));
            return launch_lines_any<float, float, true>(P, line_args(a, P->oc.D, P->nq, epb));
        }
        a.x = x;
        a.y = y;
        if (gm == kGStaged)
            return launch_lines_any<float, float, false, false, kGStaged>(P, line_args(a, P->oc.D, P->nq, epb));
        return launch_lines_any<float, float, false>(P, line_args(a, P->oc.D, P->nq, epb));
    }
    AxArgs<float, __nv_bfloat16> a = ax_args<float, __nv_bfloat16>(
        P, static_cast<const __nv_bfloat16 *>(P->G16), P->partials, P->st_in);
    if (cg) {
        a.x = P->r32;
        a.y = P->w32;
        a.p = P->p32;
        if (gm == kGRegs)
            return launch_lines_any<float, __nv_bfloat16, true, false, kGRegs>(P, line_args(a, P->oc.D, P->nq, epb));
        if (gm == kGStaged)
            return launch_lines_any<float, __nv_bfloat16, true, false, kGStaged>(P, line_args(a, P->oc.D, P->nq, epb));
        return launch_lines_any<float, __nv_bfloat16, true>(P, line_args(a, P->oc.D, P->nq, epb));
    }
    a.x = x;
    a.y = y;
    if (gm == kGRegs)
        return launch_lines_any<float, __nv_bfloat16, false, false, kGRegs>(P, line_args(a, P->oc.D, P->nq, epb));
    if (gm == kGStaged)
        return launch_lines_any<float, __nv_bfloat16, false, false, kGStaged>(P, line_args(a, P->oc.D, P->nq, epb));
    return launch_lines_any<float, __nv_bfloat16, false>(P, line_args(a, P->oc.D, P->nq, epb));
}

}  // namespace sem
