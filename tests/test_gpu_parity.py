"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances, from the arithmetic:
* geometry and local Ax: relative max-norm 1e-13.  Both sides compute in
  FP64; they differ in the derivative matrix (closed form vs barycentric,
  ~1e-15 relative), in the Jacobian route (D applied to nodal coordinates vs
  the analytic trilinear derivative) and in FMA contraction.  Each output sums
  3 (N+1) products plus the geometric 3x3 product, so rounding stays near
  1e-14 of the largest term; 1e-13 leaves an order of magnitude.
* gather-scatter, mask and the index maps: bit-exact (same additions in the
  same ascending order; integers).
* CG residual history: CG is a nonlinear recurrence, so rounding differences
  are amplified.  Measured on the oracle, a 1e-16 relative perturbation of b
  moves the 100-iteration history of the E=64, N=7 sine case by 5e-14 relative
  (amplification ~500); the GPU's operator differs by ~1e-14 relative, giving
  ~5e-12.  The bound used is 1e-9 relative per entry for histories of up to
  100 iterations from a smooth right-hand side; solves to 1e-8 from random
  data are compared by iteration count (within 2 %) and by the true residual.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _pair(oracle_mod, nx, ny, nz, N, jitter=0.05, seed=1):
    from paper_2606_12650_gb300 import Mesh
    verts = box_vertices(nx, ny, nz, jitter, seed=seed)
    return oracle_mod.Problem(nx, ny, nz, N, verts), Mesh(nx, ny, nz, N, verts)


CASES = [((1, 1, 1), 1), ((3, 2, 5), 1), ((3, 2, 5), 2), ((3, 2, 5), 3), ((5, 3, 7), 4),
         ((3, 2, 5), 5), ((3, 2, 5), 6), ((5, 3, 7), 7), ((3, 2, 5), 8), ((3, 2, 5), 9),
         ((1, 1, 1), 7), ((2, 1, 3), 9), ((7, 1, 1), 7)]


@pytest.mark.parametrize("dims,N", CASES)
def test_geometry_parity(semlib, oracle_mod, dims, N):
    P, M = _pair(oracle_mod, *dims, N, seed=N)
    G = torch.empty(P.nL * 6, dtype=torch.float64, device="cuda")
    B = torch.empty(P.nL, dtype=torch.float64, device="cuda")
    X = torch.empty(P.nL * 3, dtype=torch.float64, device="cuda")
    M.geom(G, B)
    M.nodes(X)
    assert _rel(_host(G).reshape(-1, 6), P.G) < 1e-13
    assert _rel(_host(B), P.B) < 1e-13
    assert _rel(_host(X).reshape(-1, 3), P.X) < 1e-14
    M.free()


@pytest.mark.parametrize("dims,N", CASES)
def test_ax_parity(semlib, oracle_mod, dims, N):
    P, M = _pair(oracle_mod, *dims, N, seed=10 + N)
    x = normal_field(P.nL, 20 + N)
    y_ref = P.ax_local(x)
    xd = _dev(x)
    yd = torch.full_like(xd, float("nan"))
    M.ax(xd, yd)
    assert _rel(_host(yd), y_ref) < 1e-13
    # assembled + masked operator
    yg = torch.full_like(xd, float("nan"))
    M.axg(xd, yg)
    assert _rel(_host(yg), P.apply(x)) < 1e-13
    M.free()


@pytest.mark.parametrize("dims,N", CASES)
def test_gs_mask_bit_exact(semlib, oracle_mod, dims, N):
    P, M = _pair(oracle_mod, *dims, N)
    u = normal_field(P.nL, 30 + N) * 10.0 ** (normal_field(P.nL, 31) * 3)
    ud = _dev(u)
    M.gs(ud)
    np.testing.assert_array_equal(_host(ud), P.gs(u))
    M.mask(ud)
    np.testing.assert_array_equal(_host(ud), P.mask(P.gs(u)))
    M.free()


@pytest.mark.parametrize("dims,N", [((3, 2, 5), 1), ((5, 3, 7), 4), ((4, 4, 4), 7), ((1, 1, 1), 3)])
def test_gs_map_matches_oracle_grouping(semlib, oracle_mod, dims, N):
    """The library's segments (global ids with >= 2 copies) equal the oracle's
    grouping of local indices by global id; compared as sets of sorted groups."""
    P, M = _pair(oracle_mod, *dims, N)
    assert M.nL == P.nL and M.nG == P.nG
    ptr = torch.empty(M.n_shared + 1, dtype=torch.int32, device="cuda")
    total = int((np.bincount(P.gid)[np.bincount(P.gid) >= 2]).sum())
    idx = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")
    M.gs_map(ptr, idx)
    ptr, idx = _host(ptr), _host(idx)
    assert ptr[-1] == total
    lib_groups = sorted(tuple(idx[ptr[s]:ptr[s + 1]]) for s in range(M.n_shared))
    order = np.argsort(P.gid, kind="stable")
    bounds = np.flatnonzero(np.diff(P.gid[order])) + 1
    ref_groups = sorted(tuple(g) for g in np.split(order, bounds) if len(g) >= 2)
    assert lib_groups == ref_groups
    for g in lib_groups:
        assert list(g) == sorted(g)  # copies in ascending local order
    assert M.n_masked == int(P.onbdry.sum())
    M.free()


def test_dot_rhs_and_sin(semlib, oracle_mod):
    P, M = _pair(oracle_mod, 4, 3, 2, 6)
    u, v = normal_field(P.nL, 40), normal_field(P.nL, 41)
    d = M.dot(_dev(u), _dev(v))
    assert abs(d - P.dot(u, v)) < 1e-13 * np.sqrt(P.dot(u, u) * P.dot(v, v))
    f = normal_field(P.nL, 42)
    b = torch.empty(P.nL, dtype=torch.float64, device="cuda")
    M.rhs(_dev(f), b)
    assert _rel(_host(b), P.rhs_from_source(f)) < 1e-13
    M.rhs_sin(b)
    assert _rel(_host(b), P.rhs_sin()) < 1e-13
    M.free()


def test_cg_history_config_small(semlib, oracle_mod):
    """E = 4x4x4, N = 7, jitter seed 1, sine source, 100 iterations."""
    P, M = _pair(oracle_mod, 4, 4, 4, 7, seed=1)
    b_ref = P.rhs_sin()
    x_ref, it_ref, h_ref = P.cg(b_ref, maxit=100, tol=0.0)
    b = torch.empty(P.nL, dtype=torch.float64, device="cuda")
    M.rhs_sin(b)
    x = torch.empty_like(b)
    hist = torch.zeros(101, dtype=torch.float64, device="cuda")
    it, rel = M.cg_solve(b, x, 0.0, 100, hist)
    assert it == 100 == it_ref
    h = _host(hist)
    np.testing.assert_allclose(h, h_ref, rtol=1e-9, atol=0)
    assert abs(rel - h_ref[-1] / h_ref[0]) < 1e-9 * rel
    assert _rel(_host(x), x_ref) < 1e-10
    M.free()


@pytest.mark.parametrize("dims,N,seed", [((4, 4, 4), 7, 3), ((3, 2, 5), 5, 4), ((2, 3, 2), 9, 5),
                                         ((6, 5, 4), 3, 6)])
def test_cg_to_tolerance(semlib, oracle_mod, dims, N, seed):
    P, M = _pair(oracle_mod, *dims, N, seed=seed)
    f = normal_field(P.nL, seed)
    b_ref = P.mask(P.gs(f))
    x_ref, it_ref, h_ref = P.cg(b_ref, maxit=20000, tol=1e-8)
    b = _dev(b_ref)
    x = torch.empty_like(b)
    hist = torch.zeros(20001, dtype=torch.float64, device="cuda")
    it, rel = M.cg_solve(b, x, 1e-8, 20000, hist)
    assert rel <= 1e-8
    assert abs(it - it_ref) <= max(2, 0.02 * it_ref)
    h = _host(hist)[: min(it, it_ref, 30) + 1]
    np.testing.assert_allclose(h, h_ref[: len(h)], rtol=1e-9, atol=0)
    xs = _host(x)
    assert P.true_residual(b_ref, xs) < 1.5e-8                  # oracle's operator, GPU solution
    assert abs(M.true_res(b, x) - P.true_residual(b_ref, xs)) < 1e-12
    M.free()


def test_cg_degenerate_cases(semlib, oracle_mod):
    # N = 1 on a single element: every node is on the boundary -> b = 0 -> no iterations
    P, M = _pair(oracle_mod, 1, 1, 1, 1)
    b = torch.zeros(P.nL, dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 7.0)
    it, rel = M.cg_solve(b, x, 1e-8, 100)
    assert it == 0 and rel == 0.0 and float(x.abs().max()) == 0.0
    M.free()
    # maxit = 0 returns x = 0 with the initial residual
    P, M = _pair(oracle_mod, 2, 2, 2, 3)
    b = _dev(P.rhs_sin())
    it, rel = M.cg_solve(b, torch.empty_like(b), 1e-8, 0)
    assert it == 0 and rel == 1.0
    M.free()


def test_host_mapped_end_to_end(semlib, oracle_mod):
    """Host arrays mirrored with update(to/from), kernels addressed by host pointer."""
    from paper_2606_12650_gb300 import sem
    P, M = _pair(oracle_mod, 3, 3, 3, 5, seed=8)
    b = np.ascontiguousarray(P.rhs_sin())
    x = np.zeros_like(b)
    sem.update(b, sem.SEM_TO)
    sem.update(x, sem.SEM_ALLOC)
    it, rel = M.cg_solve(b, x, 1e-10, 5000)
    sem.update(x, sem.SEM_FROM)
    sem.sync()
    x_ref, it_ref, _ = P.cg(b, maxit=5000, tol=1e-10)
    assert abs(it - it_ref) <= 2
    assert _rel(x, x_ref) < 1e-8
    # partial range copies inside the mirror
    x2 = np.zeros_like(x)
    sem.update(x2, sem.SEM_ALLOC)
    sem.update(x2, sem.SEM_FROM, 10, 20)
    sem.sync()
    sem.update(b, sem.SEM_FREE)
    sem.update(x, sem.SEM_FREE)
    sem.update(x2, sem.SEM_FREE)
    M.free()


def test_error_codes(semlib, oracle_mod):
    from paper_2606_12650_gb300 import Mesh, sem
    P, M = _pair(oracle_mod, 2, 2, 2, 3)
    xd = torch.zeros(P.nL + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.run("no_such_kernel", M.handle)
    assert e.value.code == sem.SEM_EKERNEL
    with pytest.raises(sem.SemError) as e:
        sem.run("ax", 12345, xd, xd)
    assert e.value.code == sem.SEM_EHANDLE
    with pytest.raises(sem.SemError) as e:   # 8-byte offset: not 16-byte aligned
        sem.run("ax", M.handle, sem.DevicePtr(xd.data_ptr() + 8), xd)
    assert e.value.code == sem.SEM_EARG
    with pytest.raises(sem.SemError) as e:
        sem.run("ax", M.handle, xd)
    assert e.value.code == sem.SEM_EARG
    h = np.zeros(P.nL)
    with pytest.raises(sem.SemError) as e:   # mapped argument without a mirror
        sem.run("ax", M.handle, h, xd)
    assert e.value.code == sem.SEM_ENOMAP
    with pytest.raises(sem.SemError) as e:
        sem.update(h, sem.SEM_FROM)
    assert e.value.code == sem.SEM_ENOMAP
    sem.update(h, sem.SEM_ALLOC, 0, 10)
    with pytest.raises(sem.SemError) as e:   # mirror too small for the kernel
        sem.run("ax", M.handle, h, xd)
    assert e.value.code == sem.SEM_ERANGE
    with pytest.raises(sem.SemError) as e:
        sem.update(h, sem.SEM_TO, 5, 20)
    assert e.value.code == sem.SEM_ERANGE
    sem.update(h, sem.SEM_FREE)
    with pytest.raises(sem.SemError) as e:   # double free
        sem.update(h, sem.SEM_FREE)
    assert e.value.code == sem.SEM_ENOMAP
    with pytest.raises(sem.SemError) as e:
        Mesh(2, 2, 2, 10, box_vertices(2, 2, 2, 0.0))
    assert e.value.code == sem.SEM_EARG
    bad = box_vertices(2, 2, 2, 0.0)
    bad[13] = [2.0, 2.0, 2.0]                # centre vertex pulled outside: inverted elements
    with pytest.raises(sem.SemError) as e:
        Mesh(2, 2, 2, 3, bad)
    assert e.value.code == sem.SEM_EMESH
    with pytest.raises(sem.SemError) as e:
        sem.init([])
    assert e.value.code == sem.SEM_EINIT
    M.free()
    with pytest.raises(sem.SemError) as e:
        M.handle = 999
        M.free()
    assert e.value.code == sem.SEM_EHANDLE
