// sem_pcg.cu -- Jacobi-preconditioned CG, the method of the original
// Nekbone (Section VIII-A: "Jacobi (diagonally) preconditioned conjugate
// gradient"; the paper's own C port drops the preconditioner).
//
// M = diag(A) of the assembled, masked operator.  The local diagonal of
// y = sum_ab D_a^T G_ab D_b u at node (i, j, k) of an element is
//   sum_a D_ai^2 G_rr(a,j,k) + sum_b D_bj^2 G_ss(i,b,k) + sum_c D_ck^2 G_tt(i,j,c)
//   + 2 (D_ii D_jj G_rs + D_ii D_kk G_rt + D_jj D_kk G_st)(i,j,k);
// its direct-stiffness sum is masked and inverted (0 on masked nodes).
// One PCG iteration is two kernels, like CG: the operator kernel forms
// p = M^-1 r + beta p in its prologue, and the fused gather-scatter/update
// kernel reduces both <r, M^-1 r> (beta) and <r, r> (stop test).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sem_box.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

struct DiagArgs {
    const double *G;
    double *d;
    int64_t nL;
    int nq;
    double D[kMaxQ * kMaxQ];
};

__global__ void local_diag_kernel(const DiagArgs a) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l >= a.nL) return;
    const int n = a.nq, n2 = n * n;
    const int64_t np = int64_t(n2) * n;
    const int64_t e = l / np;
    const int q = int(l - e * np);
    const int i = q % n, j = (q / n) % n, k = q / n2;
    const double *Ge = a.G + 6 * e * np;
    double v = 0.0;
    for (int m = 0; m < n; ++m) {
        v = fma(a.D[m * n + i] * a.D[m * n + i], Ge[6 * (k * n2 + j * n + m) + 0], v);
        v = fma(a.D[m * n + j] * a.D[m * n + j], Ge[6 * (k * n2 + m * n + i) + 3], v);
        v = fma(a.D[m * n + k] * a.D[m * n + k], Ge[6 * (m * n2 + j * n + i) + 5], v);
    }
    const double *g = Ge + 6 * q;
    const double Di = a.D[i * n + i], Dj = a.D[j * n + j], Dk = a.D[k * n + k];
    v += 2.0 * (Di * Dj * g[1] + Di * Dk * g[2] + Dj * Dk * g[4]);
    a.d[l] = v;
}

__global__ void invert_kernel(double *d, int64_t n) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l < n) d[l] = d[l] > 0.0 ? 1.0 / d[l] : 0.0;
}

int jacobi_prepare(Problem *P) {
    if (P->dinv) return SEM_OK;
    P->dinv = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
    if (!P->dinv) return SEM_ENOMEM;
    DiagArgs a{};
    a.G = P->G;
    a.d = P->dinv;
    a.nL = P->nL;
    a.nq = P->nq;
    for (int q = 0; q < P->nq * P->nq; ++q) a.D[q] = P->oc.D[q];
    const unsigned blocks = unsigned((P->nL + 255) / 256);
    local_diag_kernel<<<blocks, 256, 0, stream()>>>(a);
    count_launches(1);
    int rc = cuda_check(cudaGetLastError(), "local_diag_kernel");
    if (rc == SEM_OK) rc = launch_gs(P, P->dinv);
    if (rc == SEM_OK) rc = launch_mask(P, P->dinv);
    if (rc == SEM_OK) {
        invert_kernel<<<blocks, 256, 0, stream()>>>(P->dinv, P->nL);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "invert_kernel");
    }
    return rc;
}

// x = 0, p = 0, r = b; rho0 = <b, M^-1 b>, bb = <b, b> (weighted, local).
__global__ void pcg_init_kernel(const double *__restrict__ b, const double *__restrict__ c,
                                const double *__restrict__ dinv, double *__restrict__ x, double *__restrict__ r,
                                double *__restrict__ p, int64_t n, double *partials, CgState *st, int maxit,
                                double tol, double *hist) {
    __shared__ double red[32];
    double a0 = 0.0, a1 = 0.0;
    reset_group_tickets(partials);
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n; l += int64_t(gridDim.x) * blockDim.x) {
        const double bl = b[l];
        x[l] = 0.0;
        p[l] = 0.0;
        r[l] = bl;
        a0 = fma(c[l] * bl, dinv[l] * bl, a0);
        a1 = fma(c[l] * bl, bl, a1);
    }
    const double s0 = block_sum(a0, red);
    const double s1 = block_sum(a1, red);
    if (publish_partial2(s0, s1, partials, &st->ticket_dot)) {
        double rho0, bb;
        finish_partials2(partials, int(gridDim.x), &st->ticket_dot, red, &rho0, &bb);
        if (threadIdx.x == 0) {
            st->rho = rho0;
            st->rho0 = rho0;
            st->rr = bb;
            st->bb = bb;
            st->alpha = st->beta = st->pap = 0.0;
            st->tol = tol;
            st->hist = hist;
            st->iter = 0;
            st->maxit = maxit;
            st->done = (bb == 0.0 || maxit <= 0) ? 1 : 0;
            st->ticket_ax = 0;
            st->ticket_up = 0;
            if (hist) hist[0] = sqrt(bb);
        }
    }
}

template <int NQ>
__global__ void __launch_bounds__(256) pcg_update_kernel(double *__restrict__ x, double *__restrict__ r,
                                                         const double *__restrict__ p,
                                                         const double *__restrict__ w,
                                                         const double *__restrict__ dinv, int nL, BoxDims bd,
                                                         double *partials, CgState *st) {
    __shared__ double red[32];
    if (st->done) return;
    constexpr int V = UpdVec<NQ, double>::value;
    using RM = RowMap<NQ, V>;
    const double alpha = st->alpha;
    // both reductions accumulated in double-word FP32 per thread (the
    // recurrences stay FP64): GB300's FP64 pipe runs at 1/64 rate
    DwAcc rz = acc_zero<DwAcc>(), rr = acc_zero<DwAcc>();
    const int E = nL / RM::NP;
    const int ntask = RM::tasks(E);
    const int lane = threadIdx.x & 31;
    const int nwarps = int(gridDim.x * blockDim.x) >> 5;
    for (int task = int(blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarps) {
        const int l0 = RM::l0(task, lane, E);
        if (l0 >= 0) update_vec<NQ, V, double, DwAcc, true, true>(x, r, p, w, l0, bd, alpha, rz, dinv, &rr);
    }
    const double s0 = block_sum(acc_value(rz), red);
    const double s1 = block_sum(acc_value(rr), red);
    if (publish_partial2(s0, s1, partials, &st->ticket_up)) {
        double rho_new, rr_new;
        finish_partials2(partials, int(gridDim.x), &st->ticket_up, red, &rho_new, &rr_new);
        if (threadIdx.x == 0) pcg_close_iteration(st, rho_new, rr_new);
    }
}

template <int NQ>
static int launch_pcg_update_nq(const Problem *P) {
    constexpr int V = UpdVec<NQ, double>::value;
    int64_t blocks = (int64_t(RowMap<NQ, V>::tasks(int(P->E))) * 32 + 255) / 256;
    blocks = std::min<int64_t>(blocks, int64_t(sm_count()) * 8);
    pcg_update_kernel<NQ><<<unsigned(blocks), 256, 0, stream()>>>(P->x, P->r, P->p, P->w, P->dinv, int(P->nL),
                                                                  box_dims(P->nx, P->ny, P->nz), P->partials, P->st);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "pcg_update_kernel");
}

static int launch_pcg_update(const Problem *P) {
    switch (P->nq) {
        case 2: return launch_pcg_update_nq<2>(P);
        case 3: return launch_pcg_update_nq<3>(P);
        case 4: return launch_pcg_update_nq<4>(P);
        case 5: return launch_pcg_update_nq<5>(P);
        case 6: return launch_pcg_update_nq<6>(P);
        case 7: return launch_pcg_update_nq<7>(P);
        case 8: return launch_pcg_update_nq<8>(P);
        case 9: return launch_pcg_update_nq<9>(P);
        case 10: return launch_pcg_update_nq<10>(P);
        default: return set_error(SEM_EARG, "pcg: unsupported order");
    }
}

static int capture_pcg(Problem *P) {
    if (P->graph_epoch != tune_epoch()) problem_drop_graphs(P);   // operator variant changed
    if (P->graph_pcg && P->graph_stream == stream()) return SEM_OK;
    if (P->graph_pcg) {
        cudaGraphExecDestroy(P->graph_pcg);
        P->graph_pcg = nullptr;
    }
    const int K = P->nL < (1 << 20) ? 64 : 16;
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(stream(), cudaStreamCaptureModeThreadLocal), "pcg: begin capture");
    if (rc != SEM_OK) return rc;
    for (int k = 0; k < K && rc == SEM_OK; ++k) {
        rc = launch_ax_pcg(P);
        if (rc == SEM_OK) rc = launch_pcg_update(P);
    }
    count_launches(-2 * int64_t(K));
    const int rc_end = cuda_check(cudaStreamEndCapture(stream(), &g), "pcg: end capture");
    if (rc == SEM_OK) rc = rc_end;
    if (rc == SEM_OK) rc = cuda_check(cudaGraphInstantiate(&P->graph_pcg, g, 0), "pcg: instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc == SEM_OK) P->graph_stream = stream();
    P->graph_iters = K;
    return rc;
}

int pcg_solve(Problem *P, const double *b, double *x, double tol, int maxit, double *hist, int64_t *iters,
              double *rel_res) {
    if (maxit < 0) return set_error(SEM_EARG, "pcg_solve: maxit must be >= 0");
    int rc = jacobi_prepare(P);
    if (rc != SEM_OK) return rc;
    int64_t blocks = (P->nL + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    pcg_init_kernel<<<unsigned(blocks), 256, 0, stream()>>>(b, P->c, P->dinv, P->x, P->r, P->p, P->nL, P->partials,
                                                            P->st, maxit, tol, hist);
    count_launches(1);
    rc = cuda_check(cudaGetLastError(), "pcg_init_kernel");
    if (rc == SEM_OK) rc = prepare_f64_variant(P);
    if (rc == SEM_OK) rc = capture_pcg(P);
    if (rc != SEM_OK) return rc;
    const int K = P->nL < (1 << 20) ? 64 : 16;
    const int64_t max_replays = (int64_t(maxit) + K - 1) / K;
    for (int64_t rep = 0; rep < max_replays; ++rep) {
        rc = cuda_check(cudaGraphLaunch(P->graph_pcg, stream()), "pcg: graph launch");
        if (rc != SEM_OK) return rc;
        count_launches(2 * int64_t(K));
        rc = cuda_check(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                        "pcg: state read");
        if (rc == SEM_OK)
            rc = cuda_check(cudaMemcpyAsync(status_host(), status_word(), sizeof(int32_t), cudaMemcpyDeviceToHost,
                                            stream()), "pcg: status read");
        if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "pcg: sync");
        if (rc != SEM_OK) return rc;
        if (*status_host() != 0 || P->st_host->done) break;
    }
    rc = launch_x_finish(P);   // the last iteration's deferred x += alpha p
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                        "pcg: state read");
    if (rc == SEM_OK && x != P->x)
        rc = cuda_check(cudaMemcpyAsync(x, P->x, sizeof(double) * P->nL, cudaMemcpyDeviceToDevice, stream()),
                        "pcg: copy x");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "pcg: sync");
    if (rc == SEM_OK) rc = poll_status();
    if (rc != SEM_OK) return rc;
    *iters = P->st_host->iter;
    *rel_res = P->st_host->bb > 0.0 ? std::sqrt(P->st_host->rr / P->st_host->bb) : 0.0;
    return SEM_OK;
}

}  // namespace sem
