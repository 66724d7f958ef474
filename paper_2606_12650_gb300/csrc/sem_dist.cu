// sem_dist.cu -- one problem split by elements across ranks.
//
// Nekbone runs its CG under MPI with the elements divided among ranks, and
// the paper names multi-node execution as the next step for its runtime
// (Sections VIII-A, IX).  Here the E = nx ny nz box is cut into slabs of
// whole element layers along z; each rank holds one slab as an ordinary
// problem (geometry, operator, local direct-stiffness sum) plus:
//   - the interface planes it shares with the ranks below (its z0 face) and
//     above (its z1 face): for every lattice point of a plane, its local
//     copies in ascending local index (a CSR like the gs map);
//   - the Dirichlet mask of the global cube only (interface planes are not
//     masked);
//   - the global multiplicity weights: a plane point has the same number of
//     copies in the slab below and above (both slabs have the same nx, ny and
//     whole layers), so its global multiplicity is twice the local one.
// The direct-stiffness sum is the local sum, then one exchange of the plane
// partial sums with each neighbour, added lower rank's partial first (so both
// ranks hold the same bits), then the mask.  CG needs two scalar allreduces
// per iteration (<p, A p> and <r, r>).  The exchange and the allreduces are
// the caller's (sem_comm callbacks on host buffers, e.g. torch.distributed);
// everything else runs in this library's kernels.  The recurrences are those
// of cg_solve: the operator kernel in CG mode (deferred x update, p = r +
// beta p, w = A_local p, local <p, w>), then here the assembled w, r -= alpha
// w and the local <r, r>; alpha, beta and the stop test from the reduced
// scalars.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

struct DistProblem {
    Problem *P = nullptr;
    bool has_nb[2] = {false, false};      // neighbour below (z0 face), above (z1 face)
    int64_t n_plane = 0;                  // lattice points per plane: (nx N + 1)(ny N + 1)
    int32_t *plane_ptr[2] = {nullptr, nullptr};
    int32_t *plane_idx[2] = {nullptr, nullptr};
    int32_t *msk_idx = nullptr;           // local nodes on the global cube boundary
    int64_t n_mask = 0;
    double *c = nullptr;                  // 1 / global multiplicity
    double *plane_dev = nullptr;          // [2][n_plane]: one face's partial sums at a time
    double *plane_host = nullptr;         // pinned [4][n_plane]: send lo, recv lo, send hi, recv hi
};

namespace {

constexpr int kT = 256;

unsigned grid(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    return unsigned(b < 1 ? 1 : b);
}

unsigned stream_grid(int64_t n) {
    int64_t b = (n + kT - 1) / kT;
    if (b > 152 * 8) b = 152 * 8;
    return unsigned(b < 1 ? 1 : b);
}

// out[g] = u at the first local copy of plane point g (after the local sum
// every copy holds the slab's partial sum).
__global__ void plane_get_kernel(const double *__restrict__ u, const int32_t *__restrict__ ptr,
                                 const int32_t *__restrict__ idx, int64_t n, double *__restrict__ out) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g < n) out[g] = u[idx[ptr[g]]];
}

// Every copy of plane point g <- lower slab's partial + upper slab's partial.
__global__ void plane_sum_kernel(double *__restrict__ u, const int32_t *__restrict__ ptr,
                                 const int32_t *__restrict__ idx, int64_t n, const double *__restrict__ other,
                                 int own_is_lower) {
    const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const int32_t q0 = ptr[g], q1 = ptr[g + 1];
    const double own = u[idx[q0]];
    const double s = own_is_lower ? own + other[g] : other[g] + own;
    for (int32_t q = q0; q < q1; ++q) u[idx[q]] = s;
}

__global__ void dist_mask_kernel(double *__restrict__ u, const int32_t *__restrict__ idx, int64_t n) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t < n) u[idx[t]] = 0.0;
}

// x = 0, p = 0, r = b; the slab's part of <b, b>_c -> st->dot_out.
__global__ void dist_init_kernel(const double *__restrict__ b, const double *__restrict__ c,
                                 double *__restrict__ x, double *__restrict__ r, double *__restrict__ p, int64_t n,
                                 double *partials, CgState *st) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n; l += int64_t(gridDim.x) * blockDim.x) {
        const double bl = b[l];
        x[l] = 0.0;
        p[l] = 0.0;
        r[l] = bl;
        acc = fma(c[l] * bl, bl, acc);
    }
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, partials, &st->ticket_dot)) {
        const double tot = finish_partials(partials, int(gridDim.x), &st->ticket_dot, red);
        if (threadIdx.x == 0) st->dot_out = tot;
    }
}

// r -= alpha w (alpha from the state); the slab's part of <r, r>_c -> st->dot_out.
__global__ void dist_update_kernel(double *__restrict__ r, const double *__restrict__ w,
                                   const double *__restrict__ c, int64_t n, double *partials, CgState *st) {
    __shared__ double red[32];
    const double alpha = st->alpha;
    double acc = 0.0;
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n; l += int64_t(gridDim.x) * blockDim.x) {
        const double rl = fma(-alpha, w[l], r[l]);
        r[l] = rl;
        acc = fma(c[l] * rl, rl, acc);
    }
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, partials, &st->ticket_dot)) {
        const double tot = finish_partials(partials, int(gridDim.x), &st->ticket_dot, red);
        if (threadIdx.x == 0) st->dot_out = tot;
    }
}

// The slab's part of <u, v>_c -> st->dot_out.
__global__ void dist_dot_kernel(const double *__restrict__ u, const double *__restrict__ v,
                                const double *__restrict__ c, int64_t n, double *partials, CgState *st) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; l < n; l += int64_t(gridDim.x) * blockDim.x)
        acc = fma(c[l] * u[l], v[l], acc);
    const double bs = block_sum(acc, red);
    if (publish_partial(bs, partials, &st->ticket_dot)) {
        const double tot = finish_partials(partials, int(gridDim.x), &st->ticket_dot, red);
        if (threadIdx.x == 0) st->dot_out = tot;
    }
}

template <typename T>
T *upload_vec(const std::vector<T> &h, int *rc) {
    const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
    T *d = static_cast<T *>(dev_alloc(bytes));
    if (!d) {
        *rc = SEM_ENOMEM;
        return nullptr;
    }
    if (!h.empty()) {
        const int e = cuda_check(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, stream()),
                                 "dist: upload");
        if (e != SEM_OK) *rc = e;
    }
    return d;
}

// Reads one scalar of the device state into the pinned mirror.
int read_scalar(const Problem *P, const double *dev, double *host) {
    int rc = cuda_check(cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, stream()), "dist: read");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "dist: sync");
    (void)P;
    return rc;
}

int write_scalar(double *dev, double *host_pinned, double v) {
    *host_pinned = v;
    const int rc = cuda_check(cudaMemcpyAsync(dev, host_pinned, sizeof(double), cudaMemcpyHostToDevice, stream()),
                              "dist: write");
    // the pinned slot is reused by the next call: complete the copy first
    return rc == SEM_OK ? cuda_check(cudaStreamSynchronize(stream()), "dist: sync") : rc;
}

int allreduce(const sem_comm *comm, double *v, int n) {
    if (!comm || !comm->allreduce_sum) return set_error(SEM_EARG, "dist: sem_comm.allreduce_sum is missing");
    const int e = comm->allreduce_sum(comm->ctx, v, n);
    return e == 0 ? SEM_OK : set_error(SEM_ECOMM, "dist: allreduce callback failed (" + std::to_string(e) + ")");
}

}  // namespace

int dist_create(int nx, int ny, int nz, int N, const double *verts_dev, bool below, bool above, DistProblem **out) {
    *out = nullptr;
    Problem *P = nullptr;
    int rc = problem_create(nx, ny, nz, N, verts_dev, &P);
    if (rc != SEM_OK) return rc;
    rc = problem_maps(P);   // the slab's own gs map
    if (rc != SEM_OK) {
        problem_destroy(P);
        return rc;
    }
    DistProblem *D = new DistProblem();
    D->P = P;
    D->has_nb[0] = below;
    D->has_nb[1] = above;
    const int n = N + 1;
    const int64_t lx = int64_t(nx) * N + 1, ly = int64_t(ny) * N + 1, lz = int64_t(nz) * N + 1;
    D->n_plane = lx * ly;
    // lattice point of every local node, copies counted per point
    std::vector<int64_t> gid(P->nL);
    std::vector<int32_t> cnt(size_t(lx * ly * lz), 0);
    int64_t l = 0;
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex)
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i, ++l) {
                            const int64_t g = (int64_t(ex) * N + i) + lx * ((int64_t(ey) * N + j) + ly * (int64_t(ez) * N + k));
                            gid[size_t(l)] = g;
                            ++cnt[size_t(g)];
                        }
    std::vector<double> c(size_t(P->nL));
    std::vector<int32_t> msk;
    std::vector<int32_t> pptr[2], pidx[2];
    for (int f = 0; f < 2; ++f) {
        pptr[f].assign(size_t(D->n_plane) + 1, 0);
    }
    for (int64_t q = 0; q < P->nL; ++q) {
        const int64_t g = gid[size_t(q)];
        const int64_t gx = g % lx, gy = (g / lx) % ly, gz = g / (lx * ly);
        const bool lo = gz == 0, hi = gz == lz - 1;
        const bool iface = (lo && below) || (hi && above);
        c[size_t(q)] = 1.0 / double(cnt[size_t(g)] * (iface ? 2 : 1));
        if (gx == 0 || gx == lx - 1 || gy == 0 || gy == ly - 1 || (lo && !below) || (hi && !above))
            msk.push_back(int32_t(q));
        if (lo) ++pptr[0][size_t(gx + lx * gy) + 1];
        if (hi) ++pptr[1][size_t(gx + lx * gy) + 1];
    }
    for (int f = 0; f < 2; ++f) {
        for (int64_t g = 0; g < D->n_plane; ++g) pptr[f][size_t(g) + 1] += pptr[f][size_t(g)];
        pidx[f].resize(size_t(pptr[f][size_t(D->n_plane)]));
        std::vector<int32_t> fill(pptr[f].begin(), pptr[f].end() - 1);
        for (int64_t q = 0; q < P->nL; ++q) {   // ascending local index within each point
            const int64_t g = gid[size_t(q)];
            const int64_t gz = g / (lx * ly);
            if ((f == 0 && gz == 0) || (f == 1 && gz == lz - 1)) pidx[f][size_t(fill[size_t(g % (lx * ly))]++)] = int32_t(q);
        }
    }
    D->n_mask = int64_t(msk.size());
    D->msk_idx = upload_vec(msk, &rc);
    D->c = upload_vec(c, &rc);
    for (int f = 0; f < 2; ++f) {
        D->plane_ptr[f] = upload_vec(pptr[f], &rc);
        D->plane_idx[f] = upload_vec(pidx[f], &rc);
    }
    if (rc == SEM_OK) {
        D->plane_dev = static_cast<double *>(dev_alloc(sizeof(double) * 2 * size_t(D->n_plane)));
        if (!D->plane_dev) rc = SEM_ENOMEM;
    }
    if (rc == SEM_OK)
        rc = cuda_check(cudaMallocHost(&D->plane_host, sizeof(double) * 4 * size_t(D->n_plane)), "dist: pinned");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "dist: sync");
    if (rc != SEM_OK) {
        dist_destroy(D);
        return rc;
    }
    *out = D;
    return SEM_OK;
}

void dist_destroy(DistProblem *D) {
    if (!D) return;
    cudaStreamSynchronize(stream());
    if (D->P) problem_destroy(D->P);
    for (int f = 0; f < 2; ++f) {
        if (D->plane_ptr[f]) dev_free(D->plane_ptr[f]);
        if (D->plane_idx[f]) dev_free(D->plane_idx[f]);
    }
    if (D->msk_idx) dev_free(D->msk_idx);
    if (D->c) dev_free(D->c);
    if (D->plane_dev) dev_free(D->plane_dev);
    if (D->plane_host) cudaFreeHost(D->plane_host);
    delete D;
}

Problem *dist_problem(DistProblem *D) { return D->P; }

// u <- mask(QQ^T u) over all ranks: local sum, plane exchange, mask.
int dist_gs(DistProblem *D, double *u, const sem_comm *comm) {
    Problem *P = D->P;
    int rc = launch_gs(P, u);
    if (rc != SEM_OK) return rc;
    if (D->has_nb[0] || D->has_nb[1]) {
        if (!comm || !comm->exchange) return set_error(SEM_EARG, "dist: sem_comm.exchange is missing");
        const int64_t n = D->n_plane;
        double *send[2] = {D->plane_host, D->plane_host + 2 * n};
        double *recv[2] = {D->plane_host + n, D->plane_host + 3 * n};
        for (int f = 0; f < 2 && rc == SEM_OK; ++f) {
            if (!D->has_nb[f]) continue;
            plane_get_kernel<<<grid(n), kT, 0, stream()>>>(u, D->plane_ptr[f], D->plane_idx[f], n,
                                                           D->plane_dev + f * n);
            count_launches(1);
            rc = cuda_check(cudaGetLastError(), "plane_get_kernel");
            if (rc == SEM_OK)
                rc = cuda_check(cudaMemcpyAsync(send[f], D->plane_dev + f * n, sizeof(double) * size_t(n),
                                                cudaMemcpyDeviceToHost, stream()), "dist: plane out");
        }
        if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "dist: sync");
        if (rc != SEM_OK) return rc;
        const int e = comm->exchange(comm->ctx, D->has_nb[0] ? send[0] : nullptr, D->has_nb[0] ? recv[0] : nullptr,
                                     D->has_nb[1] ? send[1] : nullptr, D->has_nb[1] ? recv[1] : nullptr, n);
        if (e != 0) return set_error(SEM_ECOMM, "dist: exchange callback failed (" + std::to_string(e) + ")");
        for (int f = 0; f < 2 && rc == SEM_OK; ++f) {
            if (!D->has_nb[f]) continue;
            rc = cuda_check(cudaMemcpyAsync(D->plane_dev + f * n, recv[f], sizeof(double) * size_t(n),
                                            cudaMemcpyHostToDevice, stream()), "dist: plane in");
            if (rc != SEM_OK) break;
            // z1 face: this slab is the lower one
            plane_sum_kernel<<<grid(n), kT, 0, stream()>>>(u, D->plane_ptr[f], D->plane_idx[f], n,
                                                           D->plane_dev + f * n, f == 1 ? 1 : 0);
            count_launches(1);
            rc = cuda_check(cudaGetLastError(), "plane_sum_kernel");
        }
        if (rc != SEM_OK) return rc;
    }
    if (D->n_mask > 0) {
        dist_mask_kernel<<<grid(D->n_mask), kT, 0, stream()>>>(u, D->msk_idx, D->n_mask);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "dist_mask_kernel");
    }
    return rc;
}

int dist_dot(DistProblem *D, const double *u, const double *v, const sem_comm *comm, double *out) {
    Problem *P = D->P;
    dist_dot_kernel<<<stream_grid(P->nL), kT, 0, stream()>>>(u, v, D->c, P->nL, P->partials, P->st);
    count_launches(1);
    int rc = cuda_check(cudaGetLastError(), "dist_dot_kernel");
    double s = 0.0;
    if (rc == SEM_OK) rc = read_scalar(P, &P->st->dot_out, &P->st_host->dot_out);
    if (rc == SEM_OK) {
        s = P->st_host->dot_out;
        rc = allreduce(comm, &s, 1);
    }
    if (rc == SEM_OK) *out = s;
    return rc;
}

int dist_cg_solve(DistProblem *D, const double *b, double *x, double tol, int maxit, double *hist,
                  const sem_comm *comm, int64_t *iters, double *rel_res) {
    Problem *P = D->P;
    if (maxit < 0) return set_error(SEM_EARG, "dist_cg_solve: maxit must be >= 0");
    int rc = prepare_f64_variant(P);
    if (rc != SEM_OK) return rc;
    CgState *st = P->st, *sh = P->st_host;
    dist_init_kernel<<<stream_grid(P->nL), kT, 0, stream()>>>(b, D->c, P->x, P->r, P->p, P->nL, P->partials, st);
    count_launches(1);
    rc = cuda_check(cudaGetLastError(), "dist_init_kernel");
    if (rc == SEM_OK) rc = read_scalar(P, &st->dot_out, &sh->dot_out);
    double rho0 = sh->dot_out;
    if (rc == SEM_OK) rc = allreduce(comm, &rho0, 1);
    if (rc != SEM_OK) return rc;
    // the state the operator kernel reads: beta, alpha (deferred x update), done
    memset(sh, 0, sizeof(CgState));
    sh->rho = rho0;
    sh->rho0 = rho0;
    sh->tol = tol;
    sh->maxit = maxit;
    rc = cuda_check(cudaMemcpyAsync(st, sh, sizeof(CgState), cudaMemcpyHostToDevice, stream()), "dist: state");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "dist: sync");
    if (rc != SEM_OK) return rc;
    if (hist) hist[0] = std::sqrt(rho0);
    double rho = rho0;
    int it = 0;
    const bool run = rho0 > 0.0;
    for (int k = 1; run && k <= maxit; ++k) {
        rc = launch_ax_cg(P);   // x += alpha_{k-1} p; p = r + beta p; w = A_local p; local <p, w>
        if (rc == SEM_OK) rc = read_scalar(P, &st->pap, &sh->pap);
        double pap = sh->pap;
        if (rc == SEM_OK) rc = allreduce(comm, &pap, 1);
        if (rc != SEM_OK) return rc;
        const double alpha = rho / pap;
        rc = write_scalar(&st->alpha, &sh->alpha, alpha);
        if (rc == SEM_OK) rc = dist_gs(D, P->w, comm);
        if (rc == SEM_OK) {
            dist_update_kernel<<<stream_grid(P->nL), kT, 0, stream()>>>(P->r, P->w, D->c, P->nL, P->partials, st);
            count_launches(1);
            rc = cuda_check(cudaGetLastError(), "dist_update_kernel");
        }
        if (rc == SEM_OK) rc = read_scalar(P, &st->dot_out, &sh->dot_out);
        double rho_new = sh->dot_out;
        if (rc == SEM_OK) rc = allreduce(comm, &rho_new, 1);
        if (rc != SEM_OK) return rc;
        const double beta = rho_new / rho;
        rho = rho_new;
        rc = write_scalar(&st->beta, &sh->beta, beta);
        if (rc == SEM_OK) rc = write_scalar(&st->rho, &sh->rho, rho);
        if (rc != SEM_OK) return rc;
        it = k;
        if (hist) hist[k] = std::sqrt(rho);
        if (tol > 0.0 && std::sqrt(rho / rho0) <= tol) break;
    }
    rc = launch_x_finish(P);   // x += alpha p of the last iteration
    if (rc == SEM_OK && x != P->x)
        rc = cuda_check(cudaMemcpyAsync(x, P->x, sizeof(double) * size_t(P->nL), cudaMemcpyDeviceToDevice, stream()),
                        "dist: copy x");
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "dist: sync");
    if (rc == SEM_OK) rc = poll_status();
    if (rc != SEM_OK) return rc;
    *iters = it;
    *rel_res = rho0 > 0.0 ? std::sqrt(rho / rho0) : 0.0;
    return SEM_OK;
}

}  // namespace sem
