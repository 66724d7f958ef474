// sem_ax.cu -- FP64 instantiations of the local Poisson operator (the
// kernel itself is in sem_ax_kernel.cuh): plain y = A_local x, and the CG
// variant with the fused p-update and <p, A p> reduction.
#include "sem_ax_kernel.cuh"

namespace sem {

int prepare_ax(const Problem *Pb) { return prepare_ax_any<double, double>(Pb); }

int launch_ax(const Problem *Pb, const double *x, double *y) {
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = x;
    a.y = y;
    return launch_ax_any<double, double, false>(Pb, a);
}

int launch_ax_cg(const Problem *Pb) {
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = Pb->r;
    a.y = Pb->w;
    a.p = Pb->p;
    return launch_ax_any<double, double, true>(Pb, a);
}

int launch_ax_pcg(const Problem *Pb) {
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = Pb->r;
    a.y = Pb->w;
    a.p = Pb->p;
    a.dinv = Pb->dinv;
    return launch_ax_any<double, double, true, true>(Pb, a);
}

}  // namespace sem
