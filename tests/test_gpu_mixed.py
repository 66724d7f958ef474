"""Mixed precision (FP32 operator, FP64 iterative refinement) against the
FP64 oracle.

FP32 operator: the GPU rounds each FP64 geometric factor once to nearest
even, to FP32 or to BF16 (8 significant bits); the test applies the same
rounding to the oracle's own factors in numpy and evaluates the oracle's FP64
operator on them, with the FP32 input vector.  What remains is FP32
arithmetic (and D rounded to FP32): the FP64 kernel sits at ~45 ulp of 1.1e-16
relative max-norm against the oracle, so for FP32 (ulp 6e-8) the bound is
5e-5 relative max-norm.

Refinement: the outer residual is an FP64 recomputation, so the solution must
satisfy the oracle's own residual test at the requested tolerance (with 1.5x
slack for the different rounding of the two FP64 operators), and its error
against the oracle's FP64 CG solution is bounded by the conditioning times the
tolerance (measured on the oracle: a CG solution at tol sits within ~2 tol
of the converged one; the bound is 1e3 tol); inner iterations stay within
1.6x the FP64 CG count.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def bf16_round(a):
    """Round to nearest even with 8 significant bits (BF16 values), in FP64."""
    m, e = np.frexp(np.asarray(a, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _pair(oracle_mod, nx, ny, nz, N, seed):
    from paper_2606_12650_gb300 import Mesh
    verts = box_vertices(nx, ny, nz, 0.05, seed=seed)
    return oracle_mod.Problem(nx, ny, nz, N, verts), Mesh(nx, ny, nz, N, verts)


@pytest.mark.parametrize("gprec", [0, 1])
@pytest.mark.parametrize("dims,N", [((3, 2, 5), 1), ((3, 2, 5), 3), ((5, 3, 7), 4), ((3, 2, 5), 6),
                                    ((5, 3, 7), 7), ((2, 3, 2), 9), ((1, 1, 1), 7)])
def test_ax32_parity(semlib, oracle_mod, dims, N, gprec):
    P, M = _pair(oracle_mod, *dims, N, seed=30 + N)
    x32 = normal_field(P.nL, 60 + N).astype(np.float32)
    Gq = P.G.astype(np.float32).astype(np.float64) if gprec == 0 else bf16_round(P.G)
    y_ref = oracle_mod.ax_local(P.E, N, P.D, Gq, x32.astype(np.float64))
    xd = torch.from_numpy(x32).cuda()
    yd = torch.full_like(xd, float("nan"))
    M.ax32(xd, yd, gprec)
    torch.cuda.synchronize()
    y = yd.cpu().numpy().astype(np.float64)
    err = np.abs(y - y_ref).max() / np.abs(y_ref).max()
    assert err < 5e-5, err
    M.free()


@pytest.mark.parametrize("gprec", [0, 1])
@pytest.mark.parametrize("dims,N,seed,tol", [((4, 4, 4), 7, 3, 1e-8), ((3, 2, 5), 5, 4, 1e-10),
                                             ((2, 3, 2), 9, 5, 1e-10), ((6, 5, 4), 3, 6, 1e-8)])
def test_cg_mixed_reaches_tolerance(semlib, oracle_mod, dims, N, seed, tol, gprec):
    P, M = _pair(oracle_mod, *dims, N, seed=seed)
    b_ref = P.mask(P.gs(normal_field(P.nL, seed)))
    x_ref, it_ref, _ = P.cg(b_ref, maxit=50000, tol=1e-13)
    it_tol = P.cg(b_ref, maxit=50000, tol=tol)[1]
    b = torch.from_numpy(b_ref).cuda()
    x = torch.empty_like(b)
    hist = torch.zeros(51, dtype=torch.float64, device="cuda")
    inner, outer, res = M.cg_mixed(b, x, tol, 50, 1e-3, 100000, gprec, hist)
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    assert res <= tol
    assert P.true_residual(b_ref, xs) <= 1.5 * tol          # the oracle's operator agrees
    assert inner <= 1.6 * it_tol + 20
    h = hist.cpu().numpy()[: outer + 1]
    assert h[0] == 1.0 and abs(h[-1] - res) <= 1e-15 and np.all(np.diff(h) < 0)
    # error against the oracle's FP64 solution (converged to 1e-13)
    err = np.abs(xs - x_ref).max() / np.abs(x_ref).max()
    assert err < 1e3 * tol, err
    M.free()


def test_cg_mixed_matches_fp64_cg_on_the_small_case(semlib, oracle_mod):
    """E = 4x4x4, N = 7, sine source: mixed (BF16 G) and FP64 CG reach 1e-8."""
    P, M = _pair(oracle_mod, 4, 4, 4, 7, seed=1)
    b = torch.empty(P.nL, dtype=torch.float64, device="cuda")
    M.rhs_sin(b)
    x64 = torch.empty_like(b)
    x32 = torch.empty_like(b)
    it64, rel64 = M.cg_solve(b, x64, 1e-8, 10000)
    inner, outer, res = M.cg_mixed(b, x32, 1e-8, 20, 1e-3, 10000, 1)
    assert rel64 <= 1e-8 and res <= 1e-8
    assert M.true_res(b, x32) == pytest.approx(res, rel=1e-6)
    d = (x32 - x64).abs().max().item() / x64.abs().max().item()
    assert d < 1e-5
    M.free()


def test_cg_mixed_argument_errors(semlib, oracle_mod):
    from paper_2606_12650_gb300 import sem
    P, M = _pair(oracle_mod, 2, 2, 2, 3, seed=1)
    b = torch.zeros(P.nL, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        M.cg_mixed(b, torch.empty_like(b), 1e-8, 10, 1e-3, 100, 7)
    assert e.value.code == sem.SEM_EARG
    with pytest.raises(sem.SemError) as e:
        M.cg_mixed(b, torch.empty_like(b), 1e-8, 10, 1e-3, 0, 1)
    assert e.value.code == sem.SEM_EARG
    # zero right-hand side: nothing to do
    inner, outer, res = M.cg_mixed(b, torch.empty_like(b), 1e-8, 10, 1e-3, 100, 1)
    assert inner == 0 and outer == 0 and res == 0.0
    M.free()
