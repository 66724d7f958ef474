/*
 * sem_oracle.c -- plain, slow, FP64 CPU oracle for the spectral-element (SEM)
 * Poisson operator and the unpreconditioned conjugate-gradient solve that the
 * paper benchmarks (Nekbone, Section VIII-A: "3D Poisson equation", box domain
 * of E hexahedral elements with (N+1)^3 degrees of freedom each; the C99 port
 * has no preconditioner and runs CG for a fixed number of iterations).
 *
 * THIS FILE IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  The CUDA library shares
 * no code, header, table or helper with it.
 *
 * The paper names the operator ("the ax kernel", Section VIII-B, the most
 * expensive kernel, with N as the bound of the 1d-dof-loops) and the
 * gather-scatter kernel (Section V-B, the gs transform, whose inner j-loops are
 * order-enforced) but never writes their formulas down.  What is computed here
 * is the textbook SEM Galerkin formulation, written as plainly as possible:
 *
 *   - Gauss-Lobatto-Legendre (GLL) nodes xi_0..xi_N and weights w_j
 *   - the nodal derivative matrix D_ij = l_j'(xi_i)
 *   - a trilinear element map from 8 box vertices, Jacobian J = dx/dr
 *   - geometric factors G = W |J| J^-1 J^-T (6 symmetric entries) and
 *     mass weights B = W |J|, W = w_i w_j w_k
 *   - local Poisson action y_e = sum_ab D_a^T G_ab D_b u_e
 *   - direct-stiffness sum (QQ^T): copies of a global node are summed in
 *     ascending local index and the sum is written back to each copy
 *   - Dirichlet mask on the cube boundary
 *   - CG with the multiplicity-weighted inner product <u,v> = sum c u v,
 *     c = 1/multiplicity
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so each
 * multiply and add rounds exactly as written).
 *
 * Layout conventions (the oracle's own):
 *   local node index l = i + n*(j + n*(k + n*e)), n = N+1, i fastest
 *   element index    e = ex + nx*(ey + ny*ez)
 *   vertex index     v = a + (nx+1)*(b + (ny+1)*c), coordinates verts[3*v+d]
 *   geometric factors G[6*l + m], m = (rr, rs, rt, ss, st, tt)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Legendre polynomial P_N and its first derivative at x, by the three-term  */
/* recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1} and                  */
/* P'_{k+1} = P'_{k-1} + (2k+1) P_k.                                         */
/* ------------------------------------------------------------------------ */
static void legendre(int N, double x, double *P, double *dP)
{
    double p0 = 1.0, p1 = x;     /* P_0, P_1 */
    double d0 = 0.0, d1 = 1.0;   /* P'_0, P'_1 */
    if (N == 0) { *P = 1.0; *dP = 0.0; return; }
    for (int k = 1; k < N; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        double d2 = d0 + (2.0 * k + 1.0) * p1;
        p0 = p1; p1 = p2;
        d0 = d1; d1 = d2;
    }
    *P = p1;
    *dP = d1;
}

/* ------------------------------------------------------------------------ */
/* GLL nodes and weights.  End points are -1 and +1; the interior nodes are  */
/* the roots of P_N', found by Newton's method on P_N' starting from the     */
/* Chebyshev-Gauss-Lobatto points -cos(pi j / N).  P_N'' comes from the      */
/* Legendre equation (1-x^2) P'' = 2 x P' - N(N+1) P.  Weights are           */
/* w_j = 2 / (N (N+1) P_N(xi_j)^2).  Returns 0, or -1 for N < 1.             */
/* ------------------------------------------------------------------------ */
int orc_gll(int N, double *xi, double *w)
{
    if (N < 1) return -1;
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int j = 1; j < N; ++j) {
        double x = -cos(ORC_PI * (double)j / (double)N);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(N, x, &P, &dP);
            double d2P = (2.0 * x * dP - N * (N + 1.0) * P) / (1.0 - x * x);
            double dx = dP / d2P;
            x -= dx;
            if (fabs(dx) < 1e-15) break;
        }
        xi[j] = x;
    }
    /* ascending order (insertion sort; N is small) */
    for (int a = 1; a <= N; ++a)
        for (int b = a; b > 0 && xi[b - 1] > xi[b]; --b) {
            double t = xi[b]; xi[b] = xi[b - 1]; xi[b - 1] = t;
        }
    /* exact symmetry xi_j = -xi_{N-j} */
    for (int j = 0; j <= N / 2; ++j) {
        double a = 0.5 * (xi[N - j] - xi[j]);
        xi[j] = -a;
        xi[N - j] = a;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
    for (int j = 0; j <= N; ++j) {
        double P, dP;
        legendre(N, xi[j], &P, &dP);
        w[j] = 2.0 / (N * (N + 1.0) * P * P);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Nodal derivative matrix D[i*(N+1)+j] = l_j'(xi_i) for the Lagrange basis  */
/* on the GLL nodes (closed form in terms of P_N):                           */
/*   i != j : P_N(xi_i) / (P_N(xi_j) (xi_i - xi_j))                           */
/*   D_00 = -N(N+1)/4,  D_NN = N(N+1)/4,  other diagonal entries 0.          */
/* ------------------------------------------------------------------------ */
void orc_deriv(int N, const double *xi, double *D)
{
    int n = N + 1;
    double *P = (double *)malloc(sizeof(double) * n);
    for (int j = 0; j < n; ++j) {
        double dP;
        legendre(N, xi[j], &P[j], &dP);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v;
            if (i != j)
                v = P[i] / (P[j] * (xi[i] - xi[j]));
            else if (i == 0)
                v = -N * (N + 1.0) / 4.0;
            else if (i == N)
                v = N * (N + 1.0) / 4.0;
            else
                v = 0.0;
            D[i * n + j] = v;
        }
    free(P);
}

/* ------------------------------------------------------------------------ */
/* Nodal coordinates X[3*l + d] of every local node: the trilinear map of    */
/* the element's 8 vertices evaluated at (xi_i, xi_j, xi_k).                 */
/* ------------------------------------------------------------------------ */
void orc_nodes(int nx, int ny, int nz, int N, const double *verts,
               const double *xi, double *X)
{
    int n = N + 1;
    for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
        long e = ex + (long)nx * (ey + (long)ny * ez);
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            long l = i + n * (j + n * (k + (long)n * e));
            double r = xi[i], s = xi[j], t = xi[k];
            double hr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
            double hs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
            double ht[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
            for (int d = 0; d < 3; ++d) {
                double acc = 0.0;
                for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    long v = (ex + a) + (long)(nx + 1) * ((ey + b) + (long)(ny + 1) * (ez + c));
                    acc += verts[3 * v + d] * hr[a] * hs[b] * ht[c];
                }
                X[3 * l + d] = acc;
            }
        }
    }
}

/* The same nodal coordinates, each relative to its element's first vertex: */
/* the trilinear map applied to the vertex differences V_c - V_0.  A        */
/* translation does not change J, and coordinates formed this way carry     */
/* rounding relative to the element size h instead of to the O(1) position */
/* in the cube -- which, divided by h in the derivative and amplified by   */
/* sum_m |D_im| (~30 at N = 7), would cost ~1e-13 in G at h = 1/32.         */
void orc_nodes_rel(int nx, int ny, int nz, int N, const double *verts,
                   const double *xi, double *X)
{
    int n = N + 1;
    for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
        long e = ex + (long)nx * (ey + (long)ny * ez);
        long v0 = ex + (long)(nx + 1) * (ey + (long)(ny + 1) * ez);
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            long l = i + n * (j + n * (k + (long)n * e));
            double r = xi[i], s = xi[j], t = xi[k];
            double hr[2] = {0.5 * (1.0 - r), 0.5 * (1.0 + r)};
            double hs[2] = {0.5 * (1.0 - s), 0.5 * (1.0 + s)};
            double ht[2] = {0.5 * (1.0 - t), 0.5 * (1.0 + t)};
            for (int d = 0; d < 3; ++d) {
                double acc = 0.0;
                for (int c = 0; c < 2; ++c)
                for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    long v = (ex + a) + (long)(nx + 1) * ((ey + b) + (long)(ny + 1) * (ez + c));
                    acc += (verts[3 * v + d] - verts[3 * v0 + d]) * hr[a] * hs[b] * ht[c];
                }
                X[3 * l + d] = acc;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Geometric factors.  J_ab = dx_a/dr_b is obtained by applying D along     */
/* r, s, t to the nodal coordinates (exact for a trilinear map, whose degree */
/* per direction is 1 <= N).  The coordinates are taken relative to the      */
/* element's first node: D annihilates constants, so this is the same        */
/* derivative, without the cancellation of O(1) coordinates against O(h)    */
/* derivatives that costs digits at high N.  Then, with W = w_i w_j w_k:     */
/*   B = W |J|,   G = W |J| J^-1 J^-T  stored as (rr, rs, rt, ss, st, tt).   */
/* Returns 0, or the 1-based local index of the first node with |J| <= 0    */
/* as a negative number (an invalid mesh).                                   */
/* ------------------------------------------------------------------------ */
long orc_geometry(long E, int N, const double *X, const double *D,
                  const double *w, double *G, double *B)
{
    int n = N + 1;
    for (long e = 0; e < E; ++e)
    for (int k = 0; k < n; ++k)
    for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
        long l = i + n * (j + n * (k + (long)n * e));
        double J[3][3];   /* J[a][b] = dx_a / dr_b */
        for (int a = 0; a < 3; ++a) {
            double dr = 0.0, ds = 0.0, dt = 0.0;
            double x0 = X[3 * ((long)n * n * n * e) + a];
            for (int m = 0; m < n; ++m) {
                long lr = m + n * (j + n * (k + (long)n * e));
                long ls = i + n * (m + n * (k + (long)n * e));
                long lt = i + n * (j + n * (m + (long)n * e));
                dr += D[i * n + m] * (X[3 * lr + a] - x0);
                ds += D[j * n + m] * (X[3 * ls + a] - x0);
                dt += D[k * n + m] * (X[3 * lt + a] - x0);
            }
            J[a][0] = dr; J[a][1] = ds; J[a][2] = dt;
        }
        /* cofactors: inv[b][a] = cof[a][b] / det, inv = J^-1, inv[b][a] = dr_b/dx_a */
        double cof[3][3];
        cof[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        cof[0][1] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        cof[0][2] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        cof[1][0] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
        cof[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
        cof[1][2] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
        cof[2][0] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
        cof[2][1] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
        cof[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        double det = J[0][0] * cof[0][0] + J[0][1] * cof[0][1] + J[0][2] * cof[0][2];
        if (!(det > 0.0)) return -(l + 1);
        double inv[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                inv[b][a] = cof[a][b] / det;
        double W = w[i] * w[j] * w[k];
        double scale = W * det;
        /* G_ab = W |J| sum_c (dr_a/dx_c)(dr_b/dx_c) */
        double g[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int c = 0; c < 3; ++c) acc += inv[a][c] * inv[b][c];
                g[a][b] = scale * acc;
            }
        G[6 * l + 0] = g[0][0];
        G[6 * l + 1] = g[0][1];
        G[6 * l + 2] = g[0][2];
        G[6 * l + 3] = g[1][1];
        G[6 * l + 4] = g[1][2];
        G[6 * l + 5] = g[2][2];
        B[l] = scale;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Local Poisson action, element by element (no assembly):                  */
/*   u_r = sum_m D_im u_mjk, u_s = sum_m D_jm u_imk, u_t = sum_m D_km u_ijm  */
/*   (w_r, w_s, w_t) = G (u_r, u_s, u_t)   (G symmetric 3x3 per node)        */
/*   y_ijk = sum_m D_mi w_r,mjk + sum_m D_mj w_s,imk + sum_m D_mk w_t,ijm    */
/* Each sum runs with its index ascending.  wr/ws/wt: scratch of n^3 each.   */
/* ------------------------------------------------------------------------ */
void orc_ax_local(long E, int N, const double *D, const double *G,
                  const double *u, double *y)
{
    int n = N + 1;
    int np = n * n * n;
    double *wr = (double *)malloc(sizeof(double) * np);
    double *ws = (double *)malloc(sizeof(double) * np);
    double *wt = (double *)malloc(sizeof(double) * np);
    for (long e = 0; e < E; ++e) {
        const double *ue = u + (long)np * e;
        const double *Ge = G + 6L * np * e;
        double *ye = y + (long)np * e;
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int q = i + n * (j + n * k);
            double ur = 0.0, us = 0.0, ut = 0.0;
            for (int m = 0; m < n; ++m) {
                ur += D[i * n + m] * ue[m + n * (j + n * k)];
                us += D[j * n + m] * ue[i + n * (m + n * k)];
                ut += D[k * n + m] * ue[i + n * (j + n * m)];
            }
            const double *g = Ge + 6 * q;
            wr[q] = g[0] * ur + g[1] * us + g[2] * ut;
            ws[q] = g[1] * ur + g[3] * us + g[4] * ut;
            wt[q] = g[2] * ur + g[4] * us + g[5] * ut;
        }
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int m = 0; m < n; ++m) acc += D[m * n + i] * wr[m + n * (j + n * k)];
            for (int m = 0; m < n; ++m) acc += D[m * n + j] * ws[i + n * (m + n * k)];
            for (int m = 0; m < n; ++m) acc += D[m * n + k] * wt[i + n * (j + n * m)];
            ye[i + n * (j + n * k)] = acc;
        }
    }
    free(wr); free(ws); free(wt);
}

/* ------------------------------------------------------------------------ */
/* Global numbering of the box mesh: local node (e; i, j, k) of element      */
/* (ex, ey, ez) sits at global lattice point                                 */
/*   (gx, gy, gz) = (ex N + i, ey N + j, ez N + k)                           */
/* and gets id gx + (nx N + 1)(gy + (ny N + 1) gz).  Also flags the nodes    */
/* on the cube boundary (any lattice coordinate at 0 or its maximum).        */
/* ------------------------------------------------------------------------ */
void orc_gid(int nx, int ny, int nz, int N, int64_t *gid, uint8_t *onbdry)
{
    int n = N + 1;
    long mx = (long)nx * N, my = (long)ny * N, mz = (long)nz * N;
    for (int ez = 0; ez < nz; ++ez)
    for (int ey = 0; ey < ny; ++ey)
    for (int ex = 0; ex < nx; ++ex) {
        long e = ex + (long)nx * (ey + (long)ny * ez);
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            long l = i + n * (j + n * (k + (long)n * e));
            long gx = (long)ex * N + i, gy = (long)ey * N + j, gz = (long)ez * N + k;
            gid[l] = gx + (mx + 1) * (gy + (my + 1) * gz);
            onbdry[l] = (gx == 0 || gx == mx || gy == 0 || gy == my || gz == 0 || gz == mz);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Direct-stiffness sum QQ^T, in place.  For every global id the copies are  */
/* summed in ascending local index (the first copy starts the sum), then the */
/* sum is written to every copy.  sum/seen: scratch of nG entries.           */
/* ------------------------------------------------------------------------ */
void orc_gs(long nL, const int64_t *gid, long nG, double *u, double *sum, uint8_t *seen)
{
    memset(seen, 0, (size_t)nG);
    for (long l = 0; l < nL; ++l) {
        int64_t g = gid[l];
        if (!seen[g]) { sum[g] = u[l]; seen[g] = 1; }
        else sum[g] += u[l];
    }
    for (long l = 0; l < nL; ++l) u[l] = sum[gid[l]];
}

/* Dirichlet mask: zero every copy of a boundary node. */
void orc_mask(long nL, const uint8_t *onbdry, double *u)
{
    for (long l = 0; l < nL; ++l)
        if (onbdry[l]) u[l] = 0.0;
}

/* Multiplicity-weighted inner product sum_l c_l u_l v_l, ascending l. */
double orc_dot(long nL, const double *c, const double *u, const double *v)
{
    double acc = 0.0;
    for (long l = 0; l < nL; ++l) acc += c[l] * u[l] * v[l];
    return acc;
}

/* Full assembled, masked operator: y = mask(QQ^T(A_local u)). */
void orc_apply(long E, int N, const double *D, const double *G, long nL,
               const int64_t *gid, long nG, const uint8_t *onbdry,
               const double *u, double *y, double *sum, uint8_t *seen)
{
    orc_ax_local(E, N, D, G, u, y);
    orc_gs(nL, gid, nG, y, sum, seen);
    orc_mask(nL, onbdry, y);
}

/* ------------------------------------------------------------------------ */
/* Unpreconditioned conjugate gradient on the assembled, masked system       */
/* (Section VIII-A: the paper's C port drops Nekbone's Jacobi preconditioner */
/* and iterates CG).  Textbook recurrences:                                  */
/*   x = 0, r = b, rho = <r,r>, p = r                                        */
/*   repeat: w = A p; alpha = rho / <p,w>; x += alpha p; r -= alpha w;       */
/*           rho' = <r,r>; stop if sqrt(rho'/rho_0) <= tol or maxit reached; */
/*           beta = rho'/rho; p = r + beta p                                 */
/* <.,.> is the multiplicity-weighted product.  hist[0..iters] receives      */
/* sqrt(rho_k) (hist may be NULL).  tol <= 0 runs exactly maxit iterations.  */
/* Returns the number of iterations taken.                                   */
/* ------------------------------------------------------------------------ */
int orc_cg(long E, int N, const double *D, const double *G, long nL,
           const int64_t *gid, long nG, const uint8_t *onbdry, const double *c,
           const double *b, double *x, int maxit, double tol, double *hist)
{
    double *r = (double *)malloc(sizeof(double) * nL);
    double *p = (double *)malloc(sizeof(double) * nL);
    double *w = (double *)malloc(sizeof(double) * nL);
    double *sum = (double *)malloc(sizeof(double) * nG);
    uint8_t *seen = (uint8_t *)malloc((size_t)nG);
    for (long l = 0; l < nL; ++l) { x[l] = 0.0; r[l] = b[l]; p[l] = b[l]; }
    double rho = orc_dot(nL, c, r, r);
    double rho0 = rho;
    if (hist) hist[0] = sqrt(rho);
    int it = 0;
    if (rho0 > 0.0) {
        while (it < maxit) {
            orc_apply(E, N, D, G, nL, gid, nG, onbdry, p, w, sum, seen);
            double pw = orc_dot(nL, c, p, w);
            double alpha = rho / pw;
            for (long l = 0; l < nL; ++l) x[l] += alpha * p[l];
            for (long l = 0; l < nL; ++l) r[l] -= alpha * w[l];
            double rho_new = orc_dot(nL, c, r, r);
            ++it;
            if (hist) hist[it] = sqrt(rho_new);
            if (tol > 0.0 && sqrt(rho_new / rho0) <= tol) { rho = rho_new; break; }
            double beta = rho_new / rho;
            rho = rho_new;
            for (long l = 0; l < nL; ++l) p[l] = r[l] + beta * p[l];
        }
    }
    free(r); free(p); free(w); free(sum); free(seen);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Diagonal of the assembled, masked operator, from its definition: for    */
/* every local node q of every element, (A_e e_q)_q with e_q the unit vector */
/* at q (one local operator application per node -- slow, plain), then the */
/* direct-stiffness sum and the mask.  d: nL entries.  (Jacobi              */
/* preconditioning is the original Nekbone method, Section VIII-A.)          */
/* ------------------------------------------------------------------------ */
void orc_diag(long E, int N, const double *D, const double *G, long nL, const int64_t *gid, long nG,
              const uint8_t *onbdry, double *d)
{
    int n = N + 1;
    int np = n * n * n;
    double *u = (double *)calloc((size_t)np, sizeof(double));
    double *y = (double *)malloc(sizeof(double) * np);
    for (long e = 0; e < E; ++e) {
        for (int q = 0; q < np; ++q) {
            u[q] = 1.0;
            orc_ax_local(1, N, D, G + 6L * np * e, u, y);
            d[(long)np * e + q] = y[q];
            u[q] = 0.0;
        }
    }
    free(u); free(y);
    double *sum = (double *)malloc(sizeof(double) * nG);
    uint8_t *seen = (uint8_t *)malloc((size_t)nG);
    orc_gs(nL, gid, nG, d, sum, seen);
    orc_mask(nL, onbdry, d);
    free(sum); free(seen);
}

/* ------------------------------------------------------------------------ */
/* Jacobi-preconditioned CG (textbook):  z = M^-1 r with M = diag(A)         */
/* (zero on masked nodes), x = 0, r = b, z = M^-1 r, rho = <r,z>, p = z;    */
/* repeat: w = A p; alpha = rho/<p,w>; x += alpha p; r -= alpha w;           */
/*         z = M^-1 r; rho' = <r,z>; stop if ||r||_c/||b||_c <= tol or       */
/*         maxit; beta = rho'/rho; p = z + beta p.                           */
/* hist[k] = ||r_k||_c.  Returns the number of iterations.                   */
/* ------------------------------------------------------------------------ */
int orc_pcg(long E, int N, const double *D, const double *G, long nL,
            const int64_t *gid, long nG, const uint8_t *onbdry, const double *c,
            const double *dinv, const double *b, double *x, int maxit, double tol, double *hist)
{
    double *r = (double *)malloc(sizeof(double) * nL);
    double *z = (double *)malloc(sizeof(double) * nL);
    double *p = (double *)malloc(sizeof(double) * nL);
    double *w = (double *)malloc(sizeof(double) * nL);
    double *sum = (double *)malloc(sizeof(double) * nG);
    uint8_t *seen = (uint8_t *)malloc((size_t)nG);
    for (long l = 0; l < nL; ++l) {
        x[l] = 0.0;
        r[l] = b[l];
        z[l] = dinv[l] * r[l];
        p[l] = z[l];
    }
    double bb = orc_dot(nL, c, b, b);
    double rho = orc_dot(nL, c, r, z);
    if (hist) hist[0] = sqrt(bb);
    int it = 0;
    if (bb > 0.0) {
        while (it < maxit) {
            orc_apply(E, N, D, G, nL, gid, nG, onbdry, p, w, sum, seen);
            double pw = orc_dot(nL, c, p, w);
            double alpha = rho / pw;
            for (long l = 0; l < nL; ++l) x[l] += alpha * p[l];
            for (long l = 0; l < nL; ++l) r[l] -= alpha * w[l];
            for (long l = 0; l < nL; ++l) z[l] = dinv[l] * r[l];
            double rho_new = orc_dot(nL, c, r, z);
            double rr = orc_dot(nL, c, r, r);
            ++it;
            if (hist) hist[it] = sqrt(rr);
            if (tol > 0.0 && sqrt(rr / bb) <= tol) break;
            double beta = rho_new / rho;
            rho = rho_new;
            for (long l = 0; l < nL; ++l) p[l] = z[l] + beta * p[l];
        }
    }
    free(r); free(z); free(p); free(w); free(sum); free(seen);
    return it;
}
