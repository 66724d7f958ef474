"""Pins of the CPU oracle to facts fixed by the mathematics (no GPU).

The paper prints no worked example or value for this path (its plots are not
available), so every pin below is mathematical: closed-form quadrature rules,
library routines that reduce to a special case, exact polynomial identities,
an independent dense weak-form assembly, and manufactured solutions that the
discretisation reproduces exactly.  Each is chosen so that a plausible slip in
the oracle (a dropped geometric term, a transposed D, a wrong sign or index in
the numbering) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from paper_2606_12650_gb300.inputs import box_vertices, normal_field
from weakform import (dense_stiffness, element_stiffness, element_vertices, geometry_extended,
                      lagrange_derivs)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gll_closed_forms.json")


def _ev(expr):
    return eval(expr, {"__builtins__": {}, "sqrt": math.sqrt})


# --------------------------------------------------------------------------- GLL
def test_gll_closed_forms(oracle_mod):
    with open(GOLDEN) as fh:
        rules = json.load(fh)["rules"]
    for rule in rules:
        xi, w = oracle_mod.gll(rule["N"])
        np.testing.assert_allclose(xi, [_ev(s) for s in rule["nodes"]], rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, [_ev(s) for s in rule["weights"]], rtol=0, atol=4e-16)


@pytest.mark.parametrize("N", range(1, 17))
def test_gll_roots_of_legendre_derivative(oracle_mod, N):
    """Interior nodes = roots of P_N' (numpy's Legendre-series root finder)."""
    xi, w = oracle_mod.gll(N)
    assert xi[0] == -1.0 and xi[-1] == 1.0
    if N >= 2:
        roots = np.sort(L.Legendre.basis(N).deriv().roots().real)
        np.testing.assert_allclose(xi[1:-1], roots, rtol=0, atol=1e-13)
    # weights against the closed formula evaluated with numpy's Legendre series
    PN = L.Legendre.basis(N)(xi)
    np.testing.assert_allclose(w, 2.0 / (N * (N + 1) * PN ** 2), rtol=1e-13)
    # symmetry and total weight
    np.testing.assert_array_equal(xi, -xi[::-1])
    np.testing.assert_allclose(w, w[::-1], rtol=1e-15)
    assert abs(w.sum() - 2.0) < 1e-14


@pytest.mark.parametrize("N", range(1, 13))
def test_gll_exactness_degree(oracle_mod, N):
    """GLL with N+1 points integrates x^m exactly for m <= 2N-1, not for m = 2N."""
    xi, w = oracle_mod.gll(N)
    for m in range(0, 2 * N):
        exact = 2.0 / (m + 1) if m % 2 == 0 else 0.0
        assert abs(np.dot(w, xi ** m) - exact) < 1e-14, m
    m = 2 * N
    assert abs(np.dot(w, xi ** m) - 2.0 / (m + 1)) > 1e-8


# --------------------------------------------------------------------------- D
@pytest.mark.parametrize("N", range(1, 13))
def test_derivative_matrix(oracle_mod, N):
    xi, _ = oracle_mod.gll(N)
    D = oracle_mod.deriv(N, xi)
    # exact on monomials of degree <= N
    for m in range(0, N + 1):
        target = m * xi ** (m - 1) if m > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** m, target, rtol=0, atol=2e-13 * (m + 1) * N)
    # D 1 = 0 and centro-antisymmetry D_{N-i,N-j} = -D_{ij}
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=2e-13 * N * N)
    np.testing.assert_allclose(D[::-1, ::-1], -D, rtol=0, atol=1e-13 * N * N)
    # and against Lagrange basis derivatives built from monomial coefficients
    if N <= 8:
        np.testing.assert_allclose(D, lagrange_derivs(xi), rtol=0, atol=1e-10 * N * N)


# --------------------------------------------------------------------------- geometry
def test_geometry_undistorted_box_closed_form(oracle_mod):
    """Axis-aligned element of size (hx, hy, hz): |J| = hx hy hz / 8 and
    G = W |J| diag((2/hx)^2, (2/hy)^2, (2/hz)^2), e.g. G_rr = W hy hz / (2 hx)."""
    xs = [0.0, 0.2, 1.0]
    ys = [0.0, 0.7, 1.0]
    zs = [0.0, 0.45, 1.0]
    N = 4
    P = oracle_mod.Problem(2, 2, 2, N, box_vertices(2, 2, 2, 0.0, xs=xs, ys=ys, zs=zs))
    n = N + 1
    W = np.einsum("k,j,i->kji", P.w, P.w, P.w).ravel()
    for e in range(8):
        ex, ey, ez = e % 2, (e // 2) % 2, e // 4
        hx, hy, hz = xs[ex + 1] - xs[ex], ys[ey + 1] - ys[ey], zs[ez + 1] - zs[ez]
        sl = slice(e * n ** 3, (e + 1) * n ** 3)
        G = P.G[sl]
        np.testing.assert_allclose(P.B[sl], W * hx * hy * hz / 8, rtol=1e-13)
        np.testing.assert_allclose(G[:, 0], W * hy * hz / (2 * hx), rtol=1e-13)
        np.testing.assert_allclose(G[:, 3], W * hx * hz / (2 * hy), rtol=1e-13)
        np.testing.assert_allclose(G[:, 5], W * hx * hy / (2 * hz), rtol=1e-13)
        np.testing.assert_allclose(G[:, [1, 2, 4]], 0.0, atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_mass_sums_to_volume_under_jitter(oracle_mod, N):
    """sum B = vol = 1: GLL integrates |J| of a trilinear map exactly (degree <= 2
    per direction <= 2N-1 for N >= 2), and jitter keeps the cube."""
    P = oracle_mod.Problem(3, 2, 4, N, box_vertices(3, 2, 4, 0.05, seed=7))
    assert abs(P.B.sum() - 1.0) < 1e-13


def test_geometry_matches_analytic_jacobian(oracle_mod):
    """G and B against an analytic trilinear Jacobian (numpy inverse/det)."""
    from weakform import trilinear_jacobian
    N = 3
    nx, ny, nz = 2, 3, 2
    verts = box_vertices(nx, ny, nz, 0.05, seed=11)
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    n = N + 1
    l = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                V = element_vertices(verts, nx, ny, ex, ey, ez)
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            J = trilinear_jacobian(V, P.xi[i], P.xi[j], P.xi[k])
                            Ji = np.linalg.inv(J)
                            s = P.w[i] * P.w[j] * P.w[k] * np.linalg.det(J)
                            M = s * Ji @ Ji.T
                            ref = [M[0, 0], M[0, 1], M[0, 2], M[1, 1], M[1, 2], M[2, 2]]
                            np.testing.assert_allclose(P.G[l], ref, rtol=1e-12, atol=1e-15)
                            assert abs(P.B[l] - s) < 1e-14
                            l += 1


@pytest.mark.parametrize("N", [7, 9])
def test_geometry_extended_precision_at_benchmark_element_size(oracle_mod, N):
    """At the benchmark's element size h = 1/32 (32 x 32 x 2 jittered box),
    the FP64 geometry is within 1e-14 of max|G| of an extended-precision
    evaluation of the analytic trilinear Jacobian, and B within 1e-14 of
    max|B|.  The oracle reaches this by differentiating coordinates relative
    to each element's first vertex: from absolute O(1) coordinates the
    rounding of the position, amplified by sum_m |D_im| / h, costs ~1.5e-13."""
    nx, ny, nz = 32, 32, 2
    verts = box_vertices(nx, ny, nz, 0.05, seed=2)
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    G_ext, B_ext = geometry_extended(verts, nx, ny, nz, P.xi, P.w)
    g_err = float(np.max(np.abs(P.G - G_ext)) / np.max(np.abs(G_ext)))
    b_err = float(np.max(np.abs(P.B - B_ext)) / np.max(np.abs(B_ext)))
    assert g_err <= 1e-14, g_err
    assert b_err <= 1e-14, b_err


def test_relative_nodes_are_nodes_minus_element_origin(oracle_mod):
    """The relative nodal coordinates (the geometry's input) are the nodal
    coordinates minus each element's first vertex, and the element corners
    sit on its vertices (the trilinear map interpolates them)."""
    N, nx, ny, nz = 4, 3, 2, 2
    verts = box_vertices(nx, ny, nz, 0.05, seed=12)
    X = oracle_mod.nodes(nx, ny, nz, N, verts)
    Xr = oracle_mod.nodes_rel(nx, ny, nz, N, verts)
    n = N + 1
    npe = n ** 3
    e = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                V = element_vertices(verts, nx, ny, ex, ey, ez)
                blk = slice(e * npe, (e + 1) * npe)
                np.testing.assert_allclose(Xr[blk] + V[0, 0, 0], X[blk], rtol=0, atol=1e-15)
                Xe = X[blk].reshape(n, n, n, 3)   # [k][j][i]
                for k in (0, 1):
                    for j in (0, 1):
                        for i in (0, 1):
                            # the node at the element corner is that vertex
                            np.testing.assert_allclose(Xe[k * N, j * N, i * N], V[k, j, i], rtol=0, atol=1e-15)
                e += 1


# --------------------------------------------------------------------------- Ax
@pytest.mark.parametrize("N", [1, 2, 3, 4, 7])
def test_ax_kills_constants_before_mask(oracle_mod, N):
    P = oracle_mod.Problem(2, 3, 2, N, box_vertices(2, 3, 2, 0.05, seed=3))
    y = P.ax_local(np.ones(P.nL))
    assert np.abs(y).max() < 1e-13 * max(1.0, np.abs(P.G).max())


@pytest.mark.parametrize("N", [2, 5, 7])
def test_ax_symmetric_and_positive(oracle_mod, N):
    P = oracle_mod.Problem(2, 2, 3, N, box_vertices(2, 2, 3, 0.05, seed=5))
    x = normal_field(P.nL, 1)
    y = normal_field(P.nL, 2)
    xAy = np.dot(x, P.ax_local(y))
    yAx = np.dot(y, P.ax_local(x))
    assert abs(xAy - yAx) < 1e-13 * (abs(xAy) + np.linalg.norm(x) * np.linalg.norm(y))
    # assembled + masked operator is SPD on continuous masked vectors
    u = P.mask(P.gs(x))
    assert P.dot(u, P.apply(u)) > 0.0


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_single_affine_element_is_kronecker_sum(oracle_mod, N):
    """One axis-aligned element: A_e = a_x (B^ x B^ x A^) + a_y (B^ x A^ x B^)
    + a_z (A^ x B^ x B^), A^ = D^T W D, B^ = W, a_x = hy hz / (2 hx), ...
    (index order k, j, i with i fastest); built with numpy.kron."""
    hx, hy, hz = 0.3, 0.5, 0.8
    P = oracle_mod.Problem(1, 1, 1, N, box_vertices(1, 1, 1, 0.0, xs=[0, hx], ys=[0, hy], zs=[0, hz]))
    n = N + 1
    Wd = np.diag(P.w)
    Ah = P.D.T @ Wd @ P.D
    K = (hy * hz / (2 * hx)) * np.kron(np.kron(Wd, Wd), Ah) \
        + (hx * hz / (2 * hy)) * np.kron(np.kron(Wd, Ah), Wd) \
        + (hx * hy / (2 * hz)) * np.kron(np.kron(Ah, Wd), Wd)
    cols = np.stack([P.ax_local(np.eye(n ** 3)[c]) for c in range(n ** 3)], axis=1)
    np.testing.assert_allclose(cols, K, rtol=0, atol=1e-13 * np.abs(K).max())


@pytest.mark.parametrize("dims,N,seed", [((1, 1, 1), 3, 1), ((2, 2, 2), 2, 2),
                                         ((2, 1, 2), 3, 3), ((2, 2, 2), 3, 4)])
def test_assembled_operator_matches_dense_weak_form(oracle_mod, dims, N, seed):
    """Columns of mask-free QQ^T A_local Q against an independent dense
    weak-form assembly (analytic Jacobian, numpy Lagrange derivatives)."""
    nx, ny, nz = dims
    verts = box_vertices(nx, ny, nz, 0.05, seed=seed) if min(dims) > 1 else \
        box_vertices(nx, ny, nz, 0.0)
    if min(dims) == 1:  # no interior vertices to jitter: skew the box instead
        verts = verts + 0.1 * verts[:, [1, 2, 0]] ** 2
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    A_ref, ids = dense_stiffness(nx, ny, nz, N, verts, P.xi, P.w)
    nG = A_ref.shape[0]
    first = np.full(nG, -1)
    for l in range(P.nL - 1, -1, -1):
        first[ids[l]] = l
    A = np.empty((nG, nG))
    for g in range(nG):
        u = (ids == g).astype(float)
        A[:, g] = P.gs(P.ax_local(u))[first]
    np.testing.assert_allclose(A, A_ref, rtol=0, atol=1e-12 * np.abs(A_ref).max())


# --------------------------------------------------------------------------- gs
@pytest.mark.parametrize("dims,N", [((3, 2, 4), 1), ((2, 3, 2), 4), ((1, 1, 1), 3), ((4, 4, 4), 7)])
def test_gs_multiplicities_and_counts(oracle_mod, dims, N):
    nx, ny, nz = dims
    P = oracle_mod.Problem(nx, ny, nz, N, box_vertices(nx, ny, nz, 0.0))
    n = N + 1
    # multiplicity from position alone: a node shared along a direction iff it
    # sits on an element face in that direction that is not on the cube boundary
    mult = np.empty(P.nL)
    l = 0
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            m = 1
                            for idx, e_, ne in ((i, ex, nx), (j, ey, ny), (k, ez, nz)):
                                if (idx == 0 and e_ > 0) or (idx == N and e_ < ne - 1):
                                    m *= 2
                            mult[l] = m
                            l += 1
    np.testing.assert_array_equal(P.mult, mult)
    assert set(np.unique(P.mult)) <= {1.0, 2.0, 4.0, 8.0}
    # every global id appears; sum of multiplicities over unique ids = nL
    counts = np.bincount(P.gid, minlength=P.nG)
    assert counts.min() >= 1 and counts.sum() == P.nL
    # QQ^T 1 = multiplicity, exactly
    np.testing.assert_array_equal(P.gs(np.ones(P.nL)), P.mult)
    # QQ^T against an explicit sparse Q (numpy add.at), integer-valued data: exact
    u = np.round(normal_field(P.nL, 9) * 100)
    s = np.zeros(P.nG)
    np.add.at(s, P.gid, u)
    np.testing.assert_array_equal(P.gs(u), s[P.gid])


def test_gs_sums_in_ascending_local_order(oracle_mod):
    """Float sums depend on order: the oracle adds copies in ascending l."""
    P = oracle_mod.Problem(2, 2, 2, 2, box_vertices(2, 2, 2, 0.0))
    u = normal_field(P.nL, 4) * 10.0 ** np.arange(P.nL) % 7
    out = P.gs(u)
    for g in range(P.nG):
        ls = np.nonzero(P.gid == g)[0]
        acc = u[ls[0]]
        for l in ls[1:]:
            acc = acc + u[l]
        assert np.all(out[ls] == acc)


def test_mask_and_dot(oracle_mod):
    P = oracle_mod.Problem(3, 3, 2, 3, box_vertices(3, 3, 2, 0.05, seed=2))
    X = P.X
    on = (np.isclose(X, 0.0, atol=1e-15) | np.isclose(X, 1.0, atol=1e-15)).any(axis=1)
    np.testing.assert_array_equal(P.onbdry.astype(bool), on)
    u = P.gs(normal_field(P.nL, 3))
    # for a continuous vector the weighted local dot is the unique-node dot
    s = np.zeros(P.nG)
    s[P.gid] = u
    assert abs(P.dot(u, u) - np.dot(s, s)) < 1e-12 * np.dot(s, s)


# --------------------------------------------------------------------------- CG
@pytest.mark.parametrize("N", [3, 4, 6])
def test_cg_reproduces_manufactured_polynomial(oracle_mod, N):
    """Affine, non-uniform box; u = x(1-x) y(1-y) z(1-z), f = -Lap u.  For
    N >= 3 GLL quadrature is exact for both forms, so the discrete solution is
    the nodal interpolant of u."""
    xs, ys, zs = [0, 0.35, 1.0], [0, 0.2, 0.6, 1.0], [0, 0.5, 1.0]
    P = oracle_mod.Problem(2, 3, 2, N, box_vertices(2, 3, 2, 0.0, xs=xs, ys=ys, zs=zs))
    x, y, z = P.X.T
    u = x * (1 - x) * y * (1 - y) * z * (1 - z)
    f = 2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z) + x * (1 - x) * y * (1 - y))
    b = P.rhs_from_source(f)
    sol, it, hist = P.cg(b, maxit=2000, tol=1e-15)
    assert np.abs(sol - u).max() < 1e-12
    assert P.true_residual(b, sol) < 1e-13


@pytest.mark.parametrize("dims,N,seed", [((2, 2, 2), 2, 5), ((2, 2, 3), 3, 6)])
def test_cg_matches_dense_solve(oracle_mod, dims, N, seed):
    nx, ny, nz = dims
    verts = box_vertices(nx, ny, nz, 0.05, seed=seed)
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    A_ref, ids = dense_stiffness(nx, ny, nz, N, verts, P.xi, P.w)
    b = P.rhs_random(seed)
    interior = np.zeros(P.nG, bool)
    interior[ids[P.onbdry == 0]] = True
    bg = np.zeros(P.nG)
    bg[ids] = b
    xg = np.zeros(P.nG)
    xg[interior] = np.linalg.solve(A_ref[np.ix_(interior, interior)], bg[interior])
    sol, it, hist = P.cg(b, maxit=5000, tol=1e-14)
    np.testing.assert_allclose(sol, xg[ids], rtol=0, atol=1e-11 * np.abs(xg).max())


def test_cg_sin_error_decreases_spectrally(oracle_mod):
    """Trend only: nodal error to sin(pi x)sin(pi y)sin(pi z) falls fast with N."""
    errs = []
    for N in (2, 4, 6):
        P = oracle_mod.Problem(2, 2, 2, N, box_vertices(2, 2, 2, 0.05, seed=1))
        b = P.rhs_sin()
        sol, it, hist = P.cg(b, maxit=3000, tol=1e-13)
        x, y, z = P.X.T
        exact = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        errs.append(np.abs(sol - exact).max())
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


def test_cg_fixed_iterations_history(oracle_mod):
    """tol <= 0 runs exactly maxit iterations; the history starts at ||b||_c."""
    P = oracle_mod.Problem(4, 4, 4, 3, box_vertices(4, 4, 4, 0.05, seed=1))
    b = P.rhs_sin()
    sol, it, hist = P.cg(b, maxit=25, tol=0.0)
    assert it == 25 and len(hist) == 26
    assert abs(hist[0] - math.sqrt(P.dot(b, b))) <= 1e-15 * hist[0]
    # the recursive residual tracks the true one in the early iterations
    r = b - P.apply(sol)
    assert abs(math.sqrt(P.dot(r, r)) - hist[-1]) < 1e-8 * hist[0]


def test_input_mixes_are_near_cubic():
    """Problem mixes realise a log-uniform element count as boxes of aspect
    ratio ~1 (a prime count must not become an E x 1 x 1 box)."""
    from paper_2606_12650_gb300.inputs import batch_specs, cubic_box
    for s in batch_specs(256, seed=4):
        sides = (s["nx"], s["ny"], s["nz"])
        assert s["E"] == s["nx"] * s["ny"] * s["nz"]
        assert max(sides) - min(sides) <= 2
        assert 8 / 2 <= s["E"] <= 4096 * 1.5
    assert cubic_box(4093) == (16, 16, 16) and cubic_box(8) == (2, 2, 2)


# --------------------------------------------------------------------------- Jacobi
@pytest.mark.parametrize("dims,N,seed", [((2, 2, 2), 2, 5), ((2, 1, 2), 3, 3)])
def test_diag_is_the_dense_weak_form_diagonal(oracle_mod, dims, N, seed):
    nx, ny, nz = dims
    verts = box_vertices(nx, ny, nz, 0.05, seed=seed) if min(dims) > 1 else \
        box_vertices(nx, ny, nz, 0.0) + 0.1 * box_vertices(nx, ny, nz, 0.0)[:, [1, 2, 0]] ** 2
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    A_ref, ids = dense_stiffness(nx, ny, nz, N, verts, P.xi, P.w)
    d = P.diag()
    ref = np.diag(A_ref)[ids] * (P.onbdry == 0)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_diag_matches_closed_form(oracle_mod):
    """Local diagonal of y = D_a^T G_ab D_b u at node (i,j,k):
    sum_a D_ai^2 G_rr(a,j,k) + sum_b D_bj^2 G_ss(i,b,k) + sum_c D_ck^2 G_tt(i,j,c)
    + 2 (D_ii D_jj G_rs + D_ii D_kk G_rt + D_jj D_kk G_st)(i,j,k)."""
    N, nx, ny, nz = 4, 2, 3, 2
    P = oracle_mod.Problem(nx, ny, nz, N, box_vertices(nx, ny, nz, 0.05, seed=9))
    n = N + 1
    G = P.G.reshape(P.E, n, n, n, 6)    # [e][k][j][i][m]
    D = P.D
    loc = np.zeros((P.E, n, n, n))
    for k in range(n):
        for j in range(n):
            for i in range(n):
                v = sum(D[a, i] ** 2 * G[:, k, j, a, 0] for a in range(n))
                v = v + sum(D[b, j] ** 2 * G[:, k, b, i, 3] for b in range(n))
                v = v + sum(D[c, k] ** 2 * G[:, c, j, i, 5] for c in range(n))
                v = v + 2 * (D[i, i] * D[j, j] * G[:, k, j, i, 1] + D[i, i] * D[k, k] * G[:, k, j, i, 2]
                             + D[j, j] * D[k, k] * G[:, k, j, i, 4])
                loc[:, k, j, i] = v
    ref = P.mask(P.gs(loc.ravel()))
    np.testing.assert_allclose(P.diag(), ref, rtol=1e-13, atol=1e-15)


def test_pcg_reaches_dense_solution_in_fewer_iterations(oracle_mod):
    P = oracle_mod.Problem(3, 3, 3, 5, box_vertices(3, 3, 3, 0.05, seed=4))
    b = P.rhs_random(7)
    x_cg, it_cg, _ = P.cg(b, maxit=20000, tol=1e-10)
    x_pcg, it_pcg, hist = P.pcg(b, maxit=20000, tol=1e-10)
    assert P.true_residual(b, x_pcg) < 2e-10
    assert np.abs(x_pcg - x_cg).max() < 1e-7 * np.abs(x_cg).max()
    assert it_pcg < it_cg
    assert abs(hist[0] - np.sqrt(P.dot(b, b))) < 1e-14 * hist[0]
    # with M = I (dinv = 1 on unmasked nodes) PCG is CG
    one = (P.onbdry == 0).astype(float)
    x1, it1, _ = P.pcg(b, maxit=20000, tol=1e-10, dinv=one)
    assert it1 == it_cg and np.abs(x1 - x_cg).max() <= 1e-12 * np.abs(x_cg).max()
