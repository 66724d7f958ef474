"""Independent dense weak-form assembly used to pin the oracle (tests only).

Nothing here calls the oracle's derivative matrix, geometry or gather-scatter:
the Lagrange basis derivatives come from numpy's polynomial routines, the
element Jacobian from the analytic derivative of the trilinear vertex map, and
the global numbering from this file's own lattice formula.  The quadrature is
the GLL rule (nodes and weights passed in, pinned separately by closed forms),
i.e. the same discrete bilinear form the SEM operator evaluates:

    a(phi_p, phi_q) = sum_quad W |J| (J^-T grad_r phi_p) . (J^-T grad_r phi_q)
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import polynomial as P


def lagrange_derivs(xi):
    """Dh[a, j] = l_j'(xi_a), from explicit monomial coefficients of l_j."""
    n = len(xi)
    out = np.empty((n, n))
    for j in range(n):
        coef = P.polyfromroots(np.delete(xi, j))
        coef = coef / P.polyval(xi[j], coef)
        out[:, j] = P.polyval(xi, P.polyder(coef))
    return out


def lattice_ids(nx, ny, nz, N):
    """Global lattice id of each local node (l = i + n(j + n(k + n e)))."""
    n = N + 1
    ids = np.empty(nx * ny * nz * n ** 3, dtype=np.int64)
    mx, my = nx * N + 1, ny * N + 1
    l = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            ids[l] = (ex * N + i) + mx * ((ey * N + j) + my * (ez * N + k))
                            l += 1
    return ids


def element_vertices(verts, nx, ny, ex, ey, ez):
    """V[c, b, a, :] = vertex (ex+a, ey+b, ez+c)."""
    V = np.empty((2, 2, 2, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                v = (ex + a) + (nx + 1) * ((ey + b) + (ny + 1) * (ez + c))
                V[c, b, a] = verts[v]
    return V


def trilinear_jacobian(V, r, s, t):
    """J[a, b] = dx_a/dr_b of the trilinear map at reference point (r, s, t)."""
    h = lambda x: np.array([0.5 * (1 - x), 0.5 * (1 + x)])
    dh = np.array([-0.5, 0.5])
    hr, hs, ht = h(r), h(s), h(t)
    J = np.zeros((3, 3))
    for c in range(2):
        for b in range(2):
            for a in range(2):
                J[:, 0] += V[c, b, a] * dh[a] * hs[b] * ht[c]
                J[:, 1] += V[c, b, a] * hr[a] * dh[b] * ht[c]
                J[:, 2] += V[c, b, a] * hr[a] * hs[b] * dh[c]
    return J


def element_stiffness(V, xi, w):
    """Dense (n^3 x n^3) element stiffness with GLL quadrature."""
    n = len(xi)
    Dh = lagrange_derivs(xi)
    I = np.eye(n)
    K = np.zeros((n ** 3, n ** 3))
    for qc in range(n):
        for qb in range(n):
            for qa in range(n):
                J = trilinear_jacobian(V, xi[qa], xi[qb], xi[qc])
                det = np.linalg.det(J)
                Jinv = np.linalg.inv(J)
                W = w[qa] * w[qb] * w[qc]
                # reference gradients of all basis functions at this point,
                # basis index p = i + n(j + n k)
                gr = np.einsum("k,j,i->kji", I[qc], I[qb], Dh[qa]).ravel()
                gs = np.einsum("k,j,i->kji", I[qc], Dh[qb], I[qa]).ravel()
                gt = np.einsum("k,j,i->kji", Dh[qc], I[qb], I[qa]).ravel()
                Gref = np.stack([gr, gs, gt], axis=1)      # [p, b]  d phi_p / d r_b
                Gx = Gref @ Jinv                           # [p, c]  d phi_p / d x_c
                K += W * det * (Gx @ Gx.T)
    return K


def dense_stiffness(nx, ny, nz, N, verts, xi, w):
    """Assembled (unmasked) global stiffness over lattice ids."""
    n = N + 1
    ids = lattice_ids(nx, ny, nz, N)
    nG = (nx * N + 1) * (ny * N + 1) * (nz * N + 1)
    A = np.zeros((nG, nG))
    np_ = n ** 3
    e = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                V = element_vertices(verts, nx, ny, ex, ey, ez)
                K = element_stiffness(V, xi, w)
                g = ids[e * np_:(e + 1) * np_]
                A[np.ix_(g, g)] += K
                e += 1
    return A, ids
