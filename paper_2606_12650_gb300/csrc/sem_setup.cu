// sem_setup.cu -- problem set-up for the box-mesh SEM Poisson operator:
// quadrature rule and derivative matrix (host), direct-stiffness maps
// (host), geometric factors, nodal coordinates and right-hand sides (GPU).
//
// The paper only names these ingredients (SEM kernels relate elements,
// degrees of freedom and derivative matrices, Section III; the Nekbone box
// of E hexahedra with (N+1)^3 nodes each, Section VIII-A).  The formulas are
// the standard spectral-element ones:
//   - GLL nodes: -1, +1 and the N-1 roots of P_N', which are the zeros of
//     the degree N-1 orthogonal polynomial for the weight (1 - x^2); here
//     they are the eigenvalues of its symmetric tridiagonal Jacobi matrix,
//     found by Sturm-sequence bisection.  Weights 2 / (N(N+1) P_N(xi)^2).
//   - derivative matrix from barycentric weights:
//     D_ij = (lambda_j / lambda_i) / (xi_i - xi_j), D_ii = -sum_{j!=i} D_ij.
//   - trilinear element map; its Jacobian is differentiated analytically.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sem_device.cuh"
#include "sem_internal.h"

namespace sem {

// ---------------------------------------------------------------- quadrature
// Number of eigenvalues of the (m x m) tridiagonal matrix with zero diagonal
// and off-diagonal b[0..m-2] that are smaller than x (Sturm count).
static int sturm_count(const std::vector<double> &b, int m, double x) {
    int cnt = 0;
    double q = -x;
    if (q < 0) ++cnt;
    for (int k = 1; k < m; ++k) {
        if (q == 0.0) q = 1e-300;
        q = -x - b[k - 1] * b[k - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

static void gll_rule(int N, double *xi, double *w) {
    const int m = N - 1;  // interior nodes
    std::vector<double> b(std::max(m - 1, 0));
    for (int k = 1; k <= m - 1; ++k)
        b[k - 1] = std::sqrt(double(k) * (k + 2) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int q = 0; q < m; ++q) {
        // q-th smallest eigenvalue: smallest x with count(x) > q
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(b, m, mid) > q) hi = mid; else lo = mid;
        }
        xi[q + 1] = 0.5 * (lo + hi);
    }
    for (int q = 0; q <= N / 2; ++q) {  // enforce exact symmetry
        const double a = 0.5 * (xi[N - q] - xi[q]);
        xi[q] = -a;
        xi[N - q] = a;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int q = 0; q <= N; ++q) {
        // P_N(xi_q) by the Legendre three-term recurrence
        double pm = 1.0, pc = xi[q];
        for (int k = 1; k < N; ++k) {
            const double pn = ((2.0 * k + 1.0) * xi[q] * pc - k * pm) / (k + 1.0);
            pm = pc;
            pc = pn;
        }
        w[q] = 2.0 / (double(N) * (N + 1) * pc * pc);
    }
}

static void barycentric_derivative(int N, const double *xi, double *D) {
    const int n = N + 1;
    double lam[kMaxQ];
    for (int j = 0; j < n; ++j) {
        double prod = 1.0;
        for (int m = 0; m < n; ++m)
            if (m != j) prod *= (xi[j] - xi[m]);
        lam[j] = 1.0 / prod;
    }
    for (int i = 0; i < n; ++i) {
        double diag = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const double v = (lam[j] / lam[i]) / (xi[i] - xi[j]);
            D[i * n + j] = v;
            diag -= v;
        }
        D[i * n + i] = diag;
    }
}

void gll_rule_and_derivative(int N, double *xi, double *w, double *D) {
    gll_rule(N, xi, w);
    barycentric_derivative(N, xi, D);
}

// ---------------------------------------------------------------- geometry
struct GeomArgs {
    const double *verts;
    double *G;      // [nL][6] or nullptr
    double *B;      // [nL] or nullptr
    double *X;      // [nL][3] or nullptr
    int32_t *bad;   // first local node with |J| <= 0 (+1), atomicMin
    int64_t nL;
    int nx, ny, nq;
    double xi[kMaxQ];
    double w[kMaxQ];
};

__global__ void geom_kernel(const GeomArgs a) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l >= a.nL) return;
    const int nq = a.nq;
    const int64_t np = int64_t(nq) * nq * nq;
    const int64_t e = l / np;
    const int q = int(l - e * np);
    const int i = q % nq, j = (q / nq) % nq, k = q / (nq * nq);
    const int ex = int(e % a.nx), ey = int((e / a.nx) % a.ny), ez = int(e / (int64_t(a.nx) * a.ny));
    const double r = a.xi[i], s = a.xi[j], t = a.xi[k];
    const double hr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
    const double hs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
    const double ht[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
    const double dh[2] = {-0.5, 0.5};
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // J[d][b] = dx_d / dr_b
    double X[3] = {0, 0, 0};
    for (int cc = 0; cc < 2; ++cc)
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                const int64_t v = (ex + aa) + int64_t(a.nx + 1) * ((ey + bb) + int64_t(a.ny + 1) * (ez + cc));
                const double fr = dh[aa] * hs[bb] * ht[cc];
                const double fs = hr[aa] * dh[bb] * ht[cc];
                const double ft = hr[aa] * hs[bb] * dh[cc];
                const double f0 = hr[aa] * hs[bb] * ht[cc];
                for (int d = 0; d < 3; ++d) {
                    const double V = a.verts[3 * v + d];
                    J[d][0] += V * fr;
                    J[d][1] += V * fs;
                    J[d][2] += V * ft;
                    X[d] += V * f0;
                }
            }
    if (a.X) {
        a.X[3 * l + 0] = X[0];
        a.X[3 * l + 1] = X[1];
        a.X[3 * l + 2] = X[2];
    }
    if (!a.G) return;
    // inverse via the adjugate: Jinv[b][d] = dr_b / dx_d
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) {
        atomicMin(a.bad, int32_t(l < 0x7ffffffe ? l + 1 : 0x7ffffffe));
        return;
    }
    const double id = 1.0 / det;
    double Ji[3][3];
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    const double sc = a.w[i] * a.w[j] * a.w[k] * det;
    double g[6];
    const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int m = 0; m < 6; ++m) {
        const int A = pa[m], Bb = pb[m];
        g[m] = sc * (Ji[A][0] * Ji[Bb][0] + Ji[A][1] * Ji[Bb][1] + Ji[A][2] * Ji[Bb][2]);
    }
    double2 *G2 = reinterpret_cast<double2 *>(a.G + 6 * l);
    G2[0] = make_double2(g[0], g[1]);
    G2[1] = make_double2(g[2], g[3]);
    G2[2] = make_double2(g[4], g[5]);
    if (a.B) a.B[l] = sc;
}

static GeomArgs geom_args(const Problem *P, const double *verts) {
    GeomArgs a{};
    a.verts = verts;
    a.nL = P->nL;
    a.nx = P->nx;
    a.ny = P->ny;
    a.nq = P->nq;
    for (int q = 0; q < P->nq; ++q) {
        a.xi[q] = P->oc.xi[q];
        a.w[q] = P->oc.w[q];
    }
    return a;
}

int launch_nodes(const Problem *P, const double *verts, double *X) {
    GeomArgs a = geom_args(P, verts ? verts : P->verts);
    a.X = X;
    const int T = 256;
    geom_kernel<<<unsigned((P->nL + T - 1) / T), T, 0, stream()>>>(a);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "geom_kernel(nodes)");
}

// ---------------------------------------------------------------- right-hand sides
__global__ void rhs_sin_kernel(const double *X, const double *B, double *b, int64_t nL) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l >= nL) return;
    const double pi = 3.141592653589793238462643383279502884;
    const double x = X[3 * l], y = X[3 * l + 1], z = X[3 * l + 2];
    b[l] = B[l] * (3.0 * pi * pi * sin(pi * x) * sin(pi * y) * sin(pi * z));
}

__global__ void scale_kernel(const double *a, const double *f, double *out, int64_t n) {
    const int64_t l = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (l < n) out[l] = a[l] * f[l];
}

int launch_scale(const Problem *P, const double *a, const double *f, double *out) {
    const int T = 256;
    scale_kernel<<<unsigned((P->nL + T - 1) / T), T, 0, stream()>>>(a, f, out, P->nL);
    count_launches(1);
    return cuda_check(cudaGetLastError(), "scale_kernel");
}

int launch_rhs_sin(const Problem *P, const double *verts, double *b) {
    // nodal coordinates into the CG work vector space (x is free between solves)
    double *X = static_cast<double *>(dev_alloc(sizeof(double) * 3 * P->nL));
    if (!X) return SEM_ENOMEM;
    int rc = launch_nodes(P, verts, X);
    if (rc == SEM_OK) {
        const int T = 256;
        rhs_sin_kernel<<<unsigned((P->nL + T - 1) / T), T, 0, stream()>>>(X, P->B, b, P->nL);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "rhs_sin_kernel");
    }
    if (rc == SEM_OK) rc = launch_gs(P, b);
    if (rc == SEM_OK) rc = launch_mask(P, b);
    cudaStreamSynchronize(stream());
    dev_free(X);
    return rc;
}

// ---------------------------------------------------------------- direct-stiffness maps
// Global lattice point of local node (e; i, j, k): (ex N + i, ey N + j, ez N + k).
// Copies of one lattice point are grouped by a counting sort over the lattice
// id; within a group they keep ascending local index (stable fill order).
struct HostMaps {
    std::vector<int32_t> sh_ptr, sh_idx, msk_idx;
    std::vector<double> c;
};

static void build_maps(int nx, int ny, int nz, int N, HostMaps &M) {
    const int n = N + 1;
    const int64_t E = int64_t(nx) * ny * nz, np = int64_t(n) * n * n, nL = E * np;
    const int64_t lx = int64_t(nx) * N + 1, ly = int64_t(ny) * N + 1, lz = int64_t(nz) * N + 1;
    const int64_t nG = lx * ly * lz;
    std::vector<int64_t> gid(nL);
    std::vector<int32_t> cnt(nG, 0);
    int64_t l = 0;
    for (int ez = 0; ez < nz; ++ez)
        for (int ey = 0; ey < ny; ++ey)
            for (int ex = 0; ex < nx; ++ex)
                for (int k = 0; k < n; ++k)
                    for (int j = 0; j < n; ++j)
                        for (int i = 0; i < n; ++i, ++l) {
                            const int64_t g = (int64_t(ex) * N + i) +
                                              lx * ((int64_t(ey) * N + j) + ly * (int64_t(ez) * N + k));
                            gid[l] = g;
                            ++cnt[g];
                        }
    std::vector<int64_t> start(nG + 1, 0);
    for (int64_t g = 0; g < nG; ++g) start[g + 1] = start[g] + cnt[g];
    std::vector<int32_t> perm(nL);
    {
        std::vector<int64_t> fill(start.begin(), start.end() - 1);
        for (int64_t q = 0; q < nL; ++q) perm[fill[gid[q]]++] = int32_t(q);
    }
    M.c.resize(nL);
    for (int64_t q = 0; q < nL; ++q) M.c[q] = 1.0 / double(cnt[gid[q]]);
    M.sh_ptr.clear();
    M.sh_idx.clear();
    M.msk_idx.clear();
    M.sh_ptr.reserve(size_t(nG) + 1);
    M.sh_idx.reserve(size_t(nL));
    M.sh_ptr.push_back(0);
    for (int64_t g = 0; g < nG; ++g) {
        const int64_t gx = g % lx, gy = (g / lx) % ly, gz = g / (lx * ly);
        const bool onb = gx == 0 || gx == lx - 1 || gy == 0 || gy == ly - 1 || gz == 0 || gz == lz - 1;
        const int64_t b0 = start[g], b1 = start[g + 1];
        if (b1 - b0 >= 2) {
            for (int64_t q = b0; q < b1; ++q) M.sh_idx.push_back(perm[q]);
            M.sh_ptr.push_back(int32_t(M.sh_idx.size()));
        }
        if (onb)
            for (int64_t q = b0; q < b1; ++q) M.msk_idx.push_back(perm[q]);
    }
    std::sort(M.msk_idx.begin(), M.msk_idx.end());
}

template <typename T>
static T *upload(const std::vector<T> &h, int *rc) {
    const size_t bytes = std::max<size_t>(h.size(), 1) * sizeof(T);
    T *d = static_cast<T *>(dev_alloc(bytes));
    if (!d) {
        *rc = SEM_ENOMEM;
        return nullptr;
    }
    if (!h.empty()) {
        const int e = cuda_check(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, stream()),
                                 "upload");
        if (e != SEM_OK) *rc = e;
    }
    return d;
}

int problem_create(int nx, int ny, int nz, int N, const double *verts_dev, Problem **out, bool deferred) {
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1) return set_error(SEM_EARG, "mesh: nx, ny, nz must be >= 1");
    if (N < 1 || N > kMaxQ - 1) return set_error(SEM_EARG, "mesh: N must be in [1, 9]");
    const int64_t E = int64_t(nx) * ny * nz;
    const int64_t np = int64_t(N + 1) * (N + 1) * (N + 1);
    if (E * np >= (int64_t(1) << 31) - 1)
        return set_error(SEM_ERANGE, "mesh: E (N+1)^3 must stay below 2^31 local nodes");
    Problem *P = new Problem();
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->N = N;
    P->nq = N + 1;
    P->E = E;
    P->np = np;
    P->nL = E * np;
    P->nG = (int64_t(nx) * N + 1) * (int64_t(ny) * N + 1) * (int64_t(nz) * N + 1);
    gll_rule(N, P->oc.xi, P->oc.w);
    barycentric_derivative(N, P->oc.xi, P->oc.D);

    int rc = SEM_OK;
    const int64_t nv = int64_t(nx + 1) * (ny + 1) * (nz + 1);
    P->verts = static_cast<double *>(dev_alloc(sizeof(double) * 3 * nv));
    P->G = static_cast<double *>(dev_alloc(sizeof(double) * 6 * P->nL));
    P->B = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
    int32_t *bad = static_cast<int32_t *>(dev_alloc(sizeof(int32_t) * 4));
    P->st_host = static_cast<CgState *>(pinned_slot_alloc());
    if (!P->verts || !P->G || !P->B || !bad || !P->st_host) rc = SEM_ENOMEM;
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(P->verts, verts_dev, sizeof(double) * 3 * nv, cudaMemcpyDeviceToDevice, stream()),
                        "mesh: vertex copy");
    if (rc == SEM_OK) {
        const int32_t big = 0x7fffffff;
        rc = cuda_check(cudaMemcpyAsync(bad, &big, sizeof(int32_t), cudaMemcpyHostToDevice, stream()), "mesh: flag");
    }
    if (rc == SEM_OK) {
        GeomArgs a = geom_args(P, P->verts);
        a.G = P->G;
        a.B = P->B;
        a.bad = bad;
        const int T = 256;
        geom_kernel<<<unsigned((P->nL + T - 1) / T), T, 0, stream()>>>(a);
        count_launches(1);
        rc = cuda_check(cudaGetLastError(), "geom_kernel");
    }
    // the first non-positive Jacobian's node (or 0x7fffffff) into the pinned
    // state mirror; deferred: read by problem_check_mesh once the stream is idle
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemcpyAsync(&P->st_host->pad0, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, stream()),
                        "mesh: flag");
    if (rc == SEM_OK && !deferred) {
        rc = cuda_check(cudaStreamSynchronize(stream()), "mesh: sync");
        if (rc == SEM_OK) rc = problem_check_mesh(P);
    }
    if (bad) {
        if (deferred && rc == SEM_OK)
            P->bad_dev = bad;   // freed by problem_destroy, after the flag was read
        else
            dev_free(bad);
    }
    if (rc == SEM_OK) {
        P->x = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
        P->r = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
        P->p = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
        P->w = static_cast<double *>(dev_alloc(sizeof(double) * P->nL));
        P->partials_cap = partials_cap(P->E);
        unsigned char *pb = static_cast<unsigned char *>(dev_alloc(partials_bytes(P->partials_cap)));
        P->partials = pb ? reinterpret_cast<double *>(pb + 16) : nullptr;
        P->st = static_cast<CgState *>(dev_alloc(sizeof(CgState)));
        if (!P->x || !P->r || !P->p || !P->w || !P->partials || !P->st) rc = SEM_ENOMEM;
    }
    if (rc == SEM_OK) rc = prepare_ax(P);
    if (rc == SEM_OK) rc = cuda_check(cudaMemsetAsync(P->st, 0, sizeof(CgState), stream()), "mesh: state");
    if (rc == SEM_OK)
        rc = cuda_check(cudaMemsetAsync(group_tickets(P->partials, P->partials_cap), 0,
                                        sizeof(uint32_t) * size_t(P->partials_cap / kSumGroup), stream()),
                        "mesh: group tickets");
    if (rc == SEM_OK) {
        static_assert(sizeof(int64_t) == 8, "capacity header");
        rc = cuda_check(cudaMemcpyAsync(reinterpret_cast<unsigned char *>(P->partials) - 16, &P->partials_cap,
                                        sizeof(int64_t), cudaMemcpyHostToDevice, stream()),
                        "mesh: partials header");
    }
    if (rc == SEM_OK && !deferred) rc = cuda_check(cudaStreamSynchronize(stream()), "mesh: sync");
    if (rc != SEM_OK) {
        if (deferred) cudaStreamSynchronize(stream());   // nothing of P may still be in flight
        problem_destroy(P);
        return rc;
    }
    *out = P;
    return SEM_OK;
}

// SEM_EMESH if the geometry kernel found a non-positive Jacobian (the flag
// problem_create copied to the state mirror); the stream must be idle.
int problem_check_mesh(const Problem *P) {
    const int32_t hbad = P->st_host->pad0;
    if (hbad == 0x7fffffff) return SEM_OK;
    char msg[128];
    snprintf(msg, sizeof msg, "mesh: non-positive Jacobian at local node %d", hbad - 1);
    return set_error(SEM_EMESH, msg);
}

// Sorted-segment gather-scatter maps, mask list and multiplicity weights,
// built on the host on first use (the CG, batched and served hot paths use
// the structured box copies instead and never need them).
int problem_maps(Problem *P) {
    if (P->maps_ready) return SEM_OK;
    HostMaps M;
    build_maps(P->nx, P->ny, P->nz, P->N, M);
    int rc = SEM_OK;
    P->n_sh = int64_t(M.sh_ptr.size()) - 1;
    P->n_sh_copies = int64_t(M.sh_idx.size());
    P->n_mask = int64_t(M.msk_idx.size());
    P->sh_ptr = upload(M.sh_ptr, &rc);
    P->sh_idx = upload(M.sh_idx, &rc);
    P->msk_idx = upload(M.msk_idx, &rc);
    P->c = upload(M.c, &rc);
    if (rc == SEM_OK) rc = cuda_check(cudaStreamSynchronize(stream()), "maps: sync");
    if (rc == SEM_OK) P->maps_ready = true;
    return rc;
}

// Drops the captured CG graphs (they hold the operator variant chosen at
// capture time); the next solve captures them again.
void problem_drop_graphs(Problem *P) {
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->graph_pcg) cudaGraphExecDestroy(P->graph_pcg);
    for (auto &g : P->graph32)
        if (g) cudaGraphExecDestroy(g);
    P->graph = P->graph_pcg = nullptr;
    P->graph32[0] = P->graph32[1] = nullptr;
    P->graph_epoch = tune_epoch();
}

void problem_destroy(Problem *P) {
    if (!P) return;
    if (P->graph) cudaGraphExecDestroy(P->graph);
    if (P->graph_pcg) cudaGraphExecDestroy(P->graph_pcg);
    if (P->dinv) dev_free(P->dinv);
    if (P->bad_dev) dev_free(P->bad_dev);
    mixed_release(P);
    dw_release(P);
    if (P->partials) dev_free(reinterpret_cast<unsigned char *>(P->partials) - 16);
    double *dptrs[] = {P->verts, P->G, P->B, P->c, P->x, P->r, P->p, P->w};
    for (double *q : dptrs)
        if (q) dev_free(q);
    int32_t *iptrs[] = {P->sh_ptr, P->sh_idx, P->msk_idx};
    for (int32_t *q : iptrs)
        if (q) dev_free(q);
    if (P->st) dev_free(P->st);
    pinned_slot_free(P->st_host);
    delete P;
}

}  // namespace sem
