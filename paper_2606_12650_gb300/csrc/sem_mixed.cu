// sem_mixed.cu -- mixed-precision iterative refinement of the CG solve.
//
// Outer loop in FP64 (on the GPU): x = 0, r = b; repeat
//     solve A d = r approximately with CG in FP32 (geometric factors stored
//       in FP32 or BF16, FP32 vectors and arithmetic, FP64 dot reductions and
//       alpha/beta), stopping when its recursive residual has dropped by eta
//     x += d                          (FP64)
//     r = b - A x                     (FP64 operator, gather-scatter, mask)
//     stop when ||r||_c / ||b||_c <= tol
// The inner operator differs from A only by the rounding of G and of the
// arithmetic, so each outer step contracts the true residual by roughly
// max(eta, the operator's relative perturbation); eta is raised on the last
// step to what the target still needs (0.5 tol / current residual).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sem_box.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kThreads32 = 256;

// r32 = float(r64), d32 = 0, p32 = 0; inner rho0 = <r32, r32>_c in FP64.
__global__ void mixed_inner_init_kernel(const double *__restrict__ r64, const double *__restrict__ c,
                                        float *__restrict__ r32, float *__restrict__ d32,
                                        float *__restrict__ p32, int64_t n, double *partials, CgState *st,
                                        int maxit, double tol) {
    __shared__ double red[32];
    double acc = 0.0;
    reset_group_tickets(partials);
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n;
         l += int64_t(gridDim.x) * blockDim.x) {
        const float v = __double2float_rn(r64[l]);
        r32[l] = v;
        d32[l] = 0.f;
        p32[l] = 0.f;
        acc += c[l] * double(v) * double(v);
    }
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, partials, &st->ticket_dot)) {
        const double rho0 = finish_partials(partials, int(gridDim.x), &st->ticket_dot, red);
        if (threadIdx.x == 0) {
            st->rho = rho0;
            st->rho0 = rho0;
            st->alpha = 0.0;
            st->beta = 0.0;
            st->pap = 0.0;
            st->tol = tol;
            st->hist = nullptr;
            st->iter = 0;
            st->maxit = maxit;
            st->done = (rho0 == 0.0 || maxit <= 0) ? 1 : 0;
            st->ticket_ax = 0;
            st->ticket_up = 0;
        }
    }
}

// x64 += double(d32)
__global__ void mixed_correct_kernel(double *__restrict__ x, const float *__restrict__ d, int64_t n) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l < n) x[l] += double(d[l]);
}

static int launch_update32(const Problem *P) {
    return launch_update_rows<float, float>(P, P->d32, P->r32, P->p32, P->w32, P->st_in);
}

int mixed_prepare(Problem *P, int gprec) {
    if (gprec != kGF32 && gprec != kGBF16) return set_error(SEM_EARG, "mixed: gprec must be 0 (fp32) or 1 (bf16)");
    int rc = SEM_OK;
    void *&G = gprec == kGF32 ? P->G32 : P->G16;
    if (!G) {
        G = dev_alloc(size_t(P->nL) * 6 * (gprec == kGF32 ? 4 : 2));
        if (!G) return SEM_ENOMEM;
        rc = convert_geometry(P, gprec, G);
        if (rc != SEM_OK) return rc;
    }
    if (!P->d32) {
        const size_t vb = size_t(P->nL) * sizeof(float);
        P->d32 = static_cast<float *>(dev_alloc(vb));
        P->r32 = static_cast<float *>(dev_alloc(vb));
        P->p32 = static_cast<float *>(dev_alloc(vb));
        P->w32 = static_cast<float *>(dev_alloc(vb));
        P->st_in = static_cast<CgState *>(dev_alloc(sizeof(CgState)));
        if (!P->d32 || !P->r32 || !P->p32 || !P->w32 || !P->st_in) return SEM_ENOMEM;
        P->st_in_host = static_cast<CgState *>(pinned_slot_alloc());
        rc = P->st_in_host ? SEM_OK : SEM_ENOMEM;
        if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(P->st_in, 0, sizeof(CgState), stream()), "mixed: state");
        if (rc == SEM_OK) rc = prepare_ax32(P);
    }
    return rc;
}

void mixed_release(Problem *P) {
    for (auto &g : P->graph32)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    void *ptrs[] = {P->G32, P->G16, P->d32, P->r32, P->p32, P->w32, P->st_in};
    for (void *q : ptrs)
        if (q) dev_free(q);
    pinned_slot_free(P->st_in_host);
    P->st_in_host = nullptr;
}

static int graph32_iters_for(const Problem *P) { return P->nL < (1 << 20) ? 64 : 32; }

static int capture_inner(Problem *P, int gprec) {
    if (P->graph_epoch != tune_epoch()) problem_drop_graphs(P);   // operator variant changed
    if (P->graph32[gprec] && P->graph32_stream == stream()) return SEM_OK;
    for (auto &g : P->graph32)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    const int K = graph32_iters_for(P);
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(stream(), cudaStreamCaptureModeThreadLocal), "mixed: begin capture");
    if (rc != SEM_OK) return rc;
    for (int k = 0; k < K && rc == SEM_OK; ++k) {
        rc = launch_ax32_cg(P, gprec);
        if (rc == SEM_OK) rc = launch_update32(P);
    }
    count_launches(-2 * int64_t(K));
    const int rc_end = cuda_check(cudaStreamEndCapture(stream(), &g), "mixed: end capture");
    if (rc == SEM_OK) rc = rc_end;
    if (rc == SEM_OK) rc = cuda_check(cudaGraphInstantiate(&P->graph32[gprec], g, 0), "mixed: instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc == SEM_OK) {
        P->graph32_iters = K;
        P->graph32_stream = stream();
    }
    return rc;
}

static int read_state(CgState *host, const CgState *dev) {
    int rc = cuda_check(cudaMemcpyAsync(host, dev, sizeof(CgState), cudaMemcpyDeviceToHost, stream()), "mixed: state");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(status_host(), status_word(), sizeof(int32_t), cudaMemcpyDeviceToHost, stream()),
                        "mixed: status");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "mixed: sync");
    if (rc == SEM_OK && *status_host() != 0) rc = poll_status();
    return rc;
}

int mixed_solve(Problem *P, const double *b, double *x, double tol, int max_outer, double inner_tol,
                int inner_maxit, int gprec, int64_t *inner_iters, int64_t *outer_iters, double *rel_res,
                double *hist_outer) {
    if (max_outer < 0 || inner_maxit < 1) return set_error(SEM_EARG, "cg_mixed: bad iteration limits");
    int rc = mixed_prepare(P, gprec);
    if (rc != SEM_OK) return rc;
    rc = capture_inner(P, gprec);
    if (rc != SEM_OK) return rc;
    // x64 = 0, r64 = b, <b, b>_c (the FP64 CG initialisation)
    rc = launch_cg_init(P, b, 0, 0.0, nullptr);
    if (rc == SEM_OK) rc = read_state(P->st_host, P->st);
    if (rc != SEM_OK) return rc;
    const double bb = P->st_host->rho0;
    double rr = bb;
    int64_t inner_total = 0;
    int outer = 0;
    double res = bb > 0.0 ? 1.0 : 0.0;
    const int64_t nblk = std::min<int64_t>((P->nL + kThreads32 - 1) / kThreads32, 152 * 8);
    while (true) {
        res = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
        if (hist_outer) {
            rc = cuda_check(cudaMemcpyAsync(hist_outer + outer, &res, sizeof(double), cudaMemcpyHostToDevice, stream()),
                            "cg_mixed: history");
            if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "cg_mixed: sync");
            if (rc != SEM_OK) return rc;
        }
        if (res <= tol || outer >= max_outer) break;
        const double eta = std::min(0.5, std::max(inner_tol, 0.5 * tol / res));
        mixed_inner_init_kernel<<<unsigned(nblk), kThreads32, 0, stream()>>>(P->r, P->c, P->r32, P->d32, P->p32,
                                                                           P->nL, P->partials, P->st_in,
                                                                           inner_maxit, eta);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "mixed_inner_init_kernel");
        if (rc != SEM_OK) return rc;
        const int64_t max_replays = (int64_t(inner_maxit) + P->graph32_iters - 1) / P->graph32_iters;
        for (int64_t rep = 0; rep < max_replays; ++rep) {
            rc = cuda_check(cudaGraphLaunch(P->graph32[gprec], stream()), "mixed: graph launch");
            if (rc != SEM_OK) return rc;
            count_launches(2 * int64_t(P->graph32_iters));
            rc = read_state(P->st_in_host, P->st_in);
            if (rc != SEM_OK) return rc;
            if (P->st_in_host->done) break;
        }
        inner_total += P->st_in_host->iter;
        mixed_correct_kernel<<<unsigned((P->nL + 255) / 256), 256, 0, stream()>>>(P->x, P->d32, P->nL);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "mixed_correct_kernel");
        // true residual in FP64: r = b - mask(QQ^T(A_local x))
        if (rc == SEM_OK) rc = launch_ax(P, P->x, P->w);
        if (rc == SEM_OK) rc = launch_gs(P, P->w);
        if (rc == SEM_OK) rc = launch_mask(P, P->w);
        if (rc == SEM_OK) rc = launch_sub(P, b, P->w, P->r);
        if (rc == SEM_OK) rc = launch_dot(P, P->r, P->r);
        if (rc == SEM_OK) rc = read_state(P->st_host, P->st);
        if (rc != SEM_OK) return rc;
        rr = P->st_host->dot_out;
        ++outer;
    }
    if (x != P->x)
        rc = cuda_check(cudaMemcpyAsync(x, P->x, sizeof(double) * P->nL, cudaMemcpyDeviceToDevice, stream()),
                        "cg_mixed: copy x");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "cg_mixed: sync");
    if (rc != SEM_OK) return rc;
    *inner_iters = inner_total;
    *outer_iters = outer;
    *rel_res = res;
    return SEM_OK;
}

}  // namespace sem
