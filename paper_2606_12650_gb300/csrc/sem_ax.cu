// sem_ax.cu -- FP64 local Poisson operator: the column kernel's
// instantiations (sem_ax_kernel.cuh) -- plain y = A_local x, the CG variant
// with the fused p-update and <p, A p> reduction, the Jacobi-PCG variant --
// and the dispatch to the variant the per-order tuner chose (the line kernel
// lives in sem_ax_lines64.cu).
#include "sem_ax_kernel.cuh"

namespace sem {

int prepare_ax(const Problem *Pb) { return prepare_ax_any<double, double>(Pb); }

int launch_ax(const Problem *Pb, const double *x, double *y) {
    const TuneChoice c = tune_get(kTuneF64, Pb->nq);
    if (c.variant == kAxLines) return launch_lines64(Pb, x, y, 0, c.epb);
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = x;
    a.y = y;
    return launch_ax_any<double, double, false>(Pb, a);
}

int launch_ax_cg(const Problem *Pb) {
    const TuneChoice c = tune_get(kTuneF64, Pb->nq);
    if (c.variant == kAxLines) return launch_lines64(Pb, nullptr, nullptr, 1, c.epb);
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = Pb->r;
    a.y = Pb->w;
    a.p = Pb->p;
    a.xs = Pb->x;   // x += alpha p of the previous iteration
    return launch_ax_any<double, double, true>(Pb, a);
}

int launch_ax_pcg(const Problem *Pb) {
    const TuneChoice c = tune_get(kTuneF64, Pb->nq);
    if (c.variant == kAxLines) return launch_lines64(Pb, nullptr, nullptr, 2, c.epb);
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = Pb->r;
    a.y = Pb->w;
    a.p = Pb->p;
    a.xs = Pb->x;   // x += alpha p of the previous iteration
    a.dinv = Pb->dinv;
    return launch_ax_any<double, double, true, true>(Pb, a);
}

}  // namespace sem
