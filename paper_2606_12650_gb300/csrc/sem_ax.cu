// sem_ax.cu -- FP64 local Poisson operator: the column kernel's
// instantiations (sem_ax_kernel.cuh) -- plain y = A_local x, the CG variant
// with the fused p-update and <p, A p> reduction, the Jacobi-PCG variant --
// and the dispatch to the variant the per-order tuner chose (the line kernel
// lives in sem_ax_lines64.cu, its double-word form in sem_ax_dw.cu).
#include "sem_ax_kernel.cuh"

namespace sem {

int prepare_ax(const Problem *Pb) { return prepare_ax_any<double, double>(Pb); }

int prepare_f64_variant(Problem *P) {
    return tune_get(kTuneF64, P->nq).variant == kAxLinesDW ? dw_prepare(P) : SEM_OK;
}

// The double-word variant's factors: made on first use outside a capture
// (solves prepare them before capturing their graphs).
static int ensure_dw(const Problem *Pb) {
    if (Pb->Gdw) return SEM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const int rc = cuda_check(cudaStreamIsCapturing(stream(), &cs), "ax dw: capture status");
    if (rc != SEM_OK) return rc;
    if (cs != cudaStreamCaptureStatusNone)
        return set_error(SEM_EARG, "ax dw: double-word factors must be prepared before a capture");
    return dw_prepare(const_cast<Problem *>(Pb));
}

int launch_ax(const Problem *Pb, const double *x, double *y) {
    const TuneChoice c = tune_get(kTuneF64, Pb->nq);
    if (c.variant == kAxLinesDW) {
        const int rc = ensure_dw(Pb);
        return rc != SEM_OK ? rc : launch_lines_dw(Pb, x, y, 0, c.epb);
    }
    if (c.variant == kAxLines) return launch_lines64(Pb, x, y, 0, c.epb);
    AxArgs<double, double> a = ax_args<double, double>(Pb, Pb->G, Pb->partials, Pb->st);
    a.x = x;
    a.y = y;
    return launch_ax_any<double, double, false>(Pb, a);
}

int launch_ax_cg(const Problem *Pb) {
    const TuneChoice c = tune_get(kTuneF64, Pb->nq);
    if (c.variant == kAxLinesDW) {
        const int rc = ensure_dw(Pb);
        return rc != SEM_OK ? rc : launch_lines_dw(Pb, nullptr, nullptr, 1, c.epb);
    }
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
    if (c.variant == kAxLinesDW) {
        const int rc = ensure_dw(Pb);
        return rc != SEM_OK ? rc : launch_lines_dw(Pb, nullptr, nullptr, 2, c.epb);
    }
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
