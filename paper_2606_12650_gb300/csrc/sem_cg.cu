// sem_cg.cu -- direct-stiffness sum, Dirichlet mask, weighted dot product and
// the device-resident conjugate-gradient driver.
//
// Gather-scatter (the paper's "gs" kernel, Section V-B: an outer loop over
// global ids split across blocks and threads, and order-enforced inner loops
// over the copies).  Each thread owns one global id that has two or more
// copies; it adds the copies in ascending local index and writes the sum back
// to each.  There are no floating-point atomics, so the result does not
// depend on scheduling and matches an ascending sequential sum bit for bit.
//
// CG (Nekbone without preconditioner, Section VIII-A).  One iteration is two
// kernels:
//   1. the operator kernel in CG mode (the variant the tuner chose): the
//      previous iteration's x += alpha p, then p = r + beta p; w = A_local p;
//      <p, A p>; alpha
//   2. cg_update_class_kernel (sem_box.cuh): every local node sums the copies
//      of w of its global node in ascending local index (the direct-stiffness
//      sum), then applies r -= alpha (QQ^T w) to itself; <r, r> is
//      accumulated once per global node; the block that completes the grid
//      sum forms rho, beta, the iteration count and the stop flag.
// Moving x += alpha p into the next operator kernel (which has p in shared
// memory anyway) takes 24 of the update's 48 bytes per node off HBM and one
// FP64 operation off the update; x_finish_kernel applies the last one.
// The dot products of the paper are tree reductions (Section VIII-B, the
// unrolled reduction of Table "HIP-variable vs HIP-fixed"); here each block
// reduces in a fixed order, the last block of each group of 32 blocks sums
// the group's partials in index order and the last group sums the group sums
// (publish_grouped), so results are reproducible run to run.  Scalars
// never leave the device inside the loop: the host replays a CUDA graph of K
// iterations and polls the stop flag once per replay.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "sem_box.cuh"
#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

constexpr int kThreads = 256;

static unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return unsigned(b);
}

// ---------------------------------------------------------------- gs / mask
__global__ void gs_kernel(double *__restrict__ u, const int32_t *__restrict__ ptr,
                          const int32_t *__restrict__ idx, int64_t nseg) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= nseg) return;
    const int32_t b0 = ptr[t], b1 = ptr[t + 1];
    double s = u[idx[b0]];
    for (int32_t q = b0 + 1; q < b1; ++q) s += u[idx[q]];
    for (int32_t q = b0; q < b1; ++q) u[idx[q]] = s;
}

__global__ void mask_kernel(double *__restrict__ u, const int32_t *__restrict__ idx, int64_t n) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n) u[idx[t]] = 0.0;
}

int launch_gs(const Problem *P, double *u) {
    if (P->n_sh == 0) return SEM_OK;
    gs_kernel<<<grid_for(P->n_sh, kThreads), kThreads, 0, stream()>>>(u, P->sh_ptr, P->sh_idx, P->n_sh);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "gs_kernel");
}

int launch_mask(const Problem *P, double *u) {
    if (P->n_mask == 0) return SEM_OK;
    mask_kernel<<<grid_for(P->n_mask, kThreads), kThreads, 0, stream()>>>(u, P->msk_idx, P->n_mask);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "mask_kernel");
}

// ---------------------------------------------------------------- weighted dot
__global__ void dot_kernel(const double *__restrict__ c, const double *__restrict__ u,
                           const double *__restrict__ v, int64_t n, double *partials,
                           CgState *st) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n;
         l += int64_t(gridDim.x) * blockDim.x)
        acc = fma(c[l] * u[l], v[l], acc);
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, partials, &st->ticket_dot)) {
        const double tot = finish_partials(partials, int(gridDim.x), &st->ticket_dot, red);
        if (threadIdx.x == 0) st->dot_out = tot;
    }
}

static unsigned stream_grid(int64_t n) {
    // enough blocks to fill 152 SMs several times over, capped by the partials buffer
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return unsigned(b);
}

int launch_dot(const Problem *P, const double *u, const double *v) {
    dot_kernel<<<stream_grid(P->nL), kThreads, 0, stream()>>>(P->c, u, v, P->nL, P->partials, P->st);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "dot_kernel");
}

__global__ void sub_kernel(const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ out, int64_t n) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l < n) out[l] = a[l] - b[l];
}

int launch_sub(const Problem *P, const double *a, const double *b, double *out) {
    sub_kernel<<<grid_for(P->nL, kThreads), kThreads, 0, stream()>>>(a, b, out, P->nL);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "sub_kernel");
}

// ---------------------------------------------------------------- CG
// x = 0, p = 0, r = b; rho0 = <b, b>_c (weighted, local); scalars reset.
__global__ void cg_init_kernel(const double *__restrict__ b, const double *__restrict__ c,
                               double *__restrict__ x, double *__restrict__ r,
                               double *__restrict__ p, int64_t n, double *partials, CgState *st,
                               int maxit, double tol, double *hist) {
    __shared__ double red[32];
    double acc = 0.0;
    reset_group_tickets(partials);
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n;
         l += int64_t(gridDim.x) * blockDim.x) {
        const double bl = b[l];
        x[l] = 0.0;
        p[l] = 0.0;
        r[l] = bl;
        acc = fma(c[l] * bl, bl, acc);
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
            st->hist = hist;
            st->iter = 0;
            st->maxit = maxit;
            st->done = (rho0 == 0.0 || maxit <= 0) ? 1 : 0;
            st->ticket_ax = 0;
            st->ticket_up = 0;
            if (hist) hist[0] = sqrt(rho0);
        }
    }
}

int launch_cg_init(const Problem *P, const double *b, int maxit, double tol, double *hist) {
    cg_init_kernel<<<stream_grid(P->nL), kThreads, 0, stream()>>>(b, P->c, P->x, P->r, P->p, P->nL,
                                                                   P->partials, P->st, maxit, tol, hist);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "cg_init_kernel");
}

// The last iteration's x += alpha p: the FP64 CG operator kernel applies an
// iteration's x update at the start of the next iteration (it holds p there
// anyway); the iteration that stopped the solve has no next one.
__global__ void x_finish_kernel(double *__restrict__ x, const double *__restrict__ p, const CgState *st,
                                int64_t n) {
    const double alpha = st->alpha;
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n; l += int64_t(gridDim.x) * blockDim.x)
        x[l] = fma(alpha, p[l], x[l]);
}

int launch_x_finish(const Problem *P) {
    x_finish_kernel<<<stream_grid(P->nL), kThreads, 0, stream()>>>(P->x, P->p, P->st, P->nL);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "x_finish_kernel");
}

int launch_cg_update(const Problem *P) {
    // <r, r> accumulated in double-word FP32 per thread (sem_box.cuh)
    return launch_update_rows<double, DwAcc>(P, P->x, P->r, P->p, P->w, P->st);
}

// Iterations per captured graph: the host polls the stop flag once per replay.
static int graph_iters_for(const Problem *P) {
    // small problems are launch-bound: more iterations per replay
    return P->nL < (1 << 20) ? 64 : 16;
}

static int capture_graph(Problem *P) {
    if (P->graph_epoch != tune_epoch()) problem_drop_graphs(P);   // operator variant changed
    if (P->graph) return SEM_OK;
    const int K = graph_iters_for(P);
    cudaGraph_t g = nullptr;
    int rc = cuda_check(cudaStreamBeginCapture(stream(), cudaStreamCaptureModeThreadLocal), "cg: begin capture");
    if (rc != SEM_OK) return rc;
    for (int k = 0; k < K && rc == SEM_OK; ++k) {
        rc = launch_ax_cg(P);
        if (rc == SEM_OK) rc = launch_cg_update(P);
    }
    // launches inside a capture are counted at replay time instead
    count_launches(-2 * int64_t(K));
    const int rc_end = cuda_check(cudaStreamEndCapture(stream(), &g), "cg: end capture");
    if (rc == SEM_OK) rc = rc_end;
    if (rc == SEM_OK) rc = cuda_check(cudaGraphInstantiate(&P->graph, g, 0), "cg: instantiate");
    if (g) cudaGraphDestroy(g);
    if (rc == SEM_OK) {
        P->graph_iters = K;
        P->graph_stream = stream();
    }
    return rc;
}

int cg_solve(Problem *P, const double *b, double *x, double tol, int maxit, double *hist,
             int64_t *iters, double *rel_res) {
    if (maxit < 0) return set_error(SEM_EARG, "cg_solve: maxit must be >= 0");
    int rc = launch_cg_init(P, b, maxit, tol, hist);
    if (rc != SEM_OK) return rc;
    if (P->graph && P->graph_stream != stream()) {
        cudaGraphExecDestroy(P->graph);
        P->graph = nullptr;
    }
    rc = prepare_f64_variant(P);
    if (rc == SEM_OK) rc = capture_graph(P);
    if (rc != SEM_OK) return rc;
    // at most ceil(maxit / K) replays; the flag stops earlier replays short
    const int64_t max_replays = (int64_t(maxit) + P->graph_iters - 1) / P->graph_iters;
    for (int64_t rep = 0; rep < max_replays; ++rep) {
        rc = cuda_check(cudaGraphLaunch(P->graph, stream()), "cg: graph launch");
        if (rc != SEM_OK) return rc;
        count_launches(2 * int64_t(P->graph_iters));
        rc = cuda_check(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                        "cg: state read");
        if (rc == SEM_OK)
            rc = cuda_check(cudaMemcpyAsync(status_host(), status_word(), sizeof(int32_t),
                                            cudaMemcpyDeviceToHost, stream()),
                            "cg: status read");
        if (rc != SEM_OK) return rc;
        rc = cuda_check(cudaStreamSynchronize(stream()), "cg: sync");
        if (rc != SEM_OK) return rc;
        if (*status_host() != 0) break;
        if (P->st_host->done) break;
    }
    rc = launch_x_finish(P);
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(P->st_host, P->st, sizeof(CgState), cudaMemcpyDeviceToHost, stream()),
                        "cg: state read");
    if (rc == SEM_OK && x != P->x)
        rc = cuda_check(cudaMemcpyAsync(x, P->x, sizeof(double) * P->nL, cudaMemcpyDeviceToDevice, stream()),
                        "cg: copy x");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "cg: sync");
    if (rc != SEM_OK) return rc;
    rc = poll_status();
    if (rc != SEM_OK) return rc;
    *iters = P->st_host->iter;
    *rel_res = P->st_host->rho0 > 0.0 ? std::sqrt(P->st_host->rho / P->st_host->rho0) : 0.0;
    return SEM_OK;
}

}  // namespace sem
