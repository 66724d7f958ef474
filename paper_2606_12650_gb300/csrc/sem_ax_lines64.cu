// sem_ax_lines64.cu -- FP64 instantiations of the line kernel
// (sem_ax_lines.cuh): plain y = A_local x, the CG operator and the
// Jacobi-PCG operator, for every order, with the elements per block chosen at
// launch.
#include "sem_ax_lines.cuh"

namespace sem {

bool lines_epb_ok(int nq, int epb, size_t elem_bytes, int g_stage_bytes) {
    if (nq < 2 || nq > kMaxQ || epb < 1 || line_threads(nq, epb) == 0) return false;
    return LineShape::smem(nq, epb, int(elem_bytes), g_stage_bytes) <= size_t(200) * 1024;
}

int launch_lines64(const Problem *P, const double *x, double *y, int mode, int epb) {
    if (!lines_epb_ok(P->nq, epb, sizeof(double))) return set_error(SEM_EARG, "ax lines: bad elements per block");
    AxArgs<double, double> a = ax_args<double, double>(P, P->G, P->partials, P->st);
    if (mode == 0) {
        a.x = x;
        a.y = y;
        return launch_lines_any<double, double, false>(P, line_args(a, P->oc.D, P->nq, epb));
    }
    a.x = P->r;
    a.y = P->w;
    a.p = P->p;
    a.xs = P->x;   // x += alpha p of the previous iteration
    if (mode == 1) return launch_lines_any<double, double, true>(P, line_args(a, P->oc.D, P->nq, epb));
    a.dinv = P->dinv;
    return launch_lines_any<double, double, true, true>(P, line_args(a, P->oc.D, P->nq, epb));
}

}  // namespace sem
