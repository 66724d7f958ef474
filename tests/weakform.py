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


def geometry_extended(verts, nx, ny, nz, xi, w):
    """G [nL, 6] and B [nL] of every local node in extended precision.

    The Jacobian is the analytic derivative of the trilinear vertex map (no
    derivative matrix, no nodal coordinates), evaluated in ``np.longdouble``
    (64-bit significand on x86, IEEE quad on Arm) from the FP64 vertices; the
    inverse is the adjugate over the determinant.  The result carries ~11 more
    bits than an FP64 evaluation, so it measures the FP64 geometry's rounding.
    """
    Lg = np.longdouble
    n = len(xi)
    xi = np.asarray(xi).astype(Lg)
    w = np.asarray(w).astype(Lg)
    V = np.asarray(verts).astype(Lg).reshape(nz + 1, ny + 1, nx + 1, 3)
    hf = np.stack([(1 - xi) / 2, (1 + xi) / 2])                 # hat functions [a, node]
    dh = np.stack([np.full(n, Lg(-0.5)), np.full(n, Lg(0.5))])  # their derivatives
    J = np.zeros((nz, ny, nx, n, n, n, 3, 3), dtype=Lg)          # [..., k, j, i, x_d, r_b]
    for c in range(2):
        for b in range(2):
            for a in range(2):
                Vc = V[c:c + nz, b:b + ny, a:a + nx][:, :, :, None, None, None, :]
                for col, f in enumerate((np.einsum("k,j,i->kji", hf[c], hf[b], dh[a]),
                                         np.einsum("k,j,i->kji", hf[c], dh[b], hf[a]),
                                         np.einsum("k,j,i->kji", dh[c], hf[b], hf[a]))):
                    J[..., :, col] += Vc * f[None, None, None, :, :, :, None]
    cof = np.empty_like(J)
    for r in range(3):
        for s in range(3):
            r1, r2 = [q for q in range(3) if q != r]
            s1, s2 = [q for q in range(3) if q != s]
            sign = 1 if (r + s) % 2 == 0 else -1
            cof[..., r, s] = sign * (J[..., r1, s1] * J[..., r2, s2] - J[..., r1, s2] * J[..., r2, s1])
    det = np.einsum("...b,...b->...", J[..., 0, :], cof[..., 0, :])
    Jinv = np.swapaxes(cof, -1, -2) / det[..., None, None]
    W = np.einsum("k,j,i->kji", w, w, w)[None, None, None]
    M = np.einsum("...ab,...cb->...ac", Jinv, Jinv) * (W * det)[..., None, None]
    G = np.stack([M[..., 0, 0], M[..., 0, 1], M[..., 0, 2], M[..., 1, 1], M[..., 1, 2], M[..., 2, 2]], -1)
    return G.reshape(-1, 6), (W * det).reshape(-1)
