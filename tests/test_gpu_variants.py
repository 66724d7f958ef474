"""Operator variants and the per-order tuner.

Every variant computes the same map, so each is held to the bar of the
default one: FP64 local and assembled operator within 1e-13 (relative max
norm) of the oracle for every order, including odd N+1 (a middle node in the
even-odd split) and blocks whose last element group is ragged; CG and
Jacobi-PCG residual histories within rtol 1e-9 of the oracle's; FP32
operator within 5e-5 of the oracle evaluated on the same rounded geometric
factors.  The double-word variant (the FP64 operator in pairs of FP32
numbers, ~48 significant bits) is held to the same FP64 bars; its CG
histories get the absolute floor scaled to its rounding unit (2^-48 instead
of 2^-53 of ||b||).  The tuner returns one timing per candidate, keeps the fastest, and
its table survives a save/load round trip; changing the variant makes
captured CG graphs be captured again.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F64, F32G32, F32G16 = 0, 1, 2
COLUMNS, LINES, PERSISTENT, LINES_PF, LINES_ST, LINES_DW = 0, 1, 2, 3, 4, 5


def bf16_round(a):
    m, e = np.frexp(np.asarray(a, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


class variant:
    """Use (variant, epb) for (kind, N) inside a with-block, then restore."""

    def __init__(self, kind, N, v, epb=0):
        self.key, self.new = (kind, N), (v, epb)

    def __enter__(self):
        from paper_2606_12650_gb300 import sem
        self.old = sem.autotune_get(*self.key)
        sem.autotune_set(*self.key, *self.new)

    def __exit__(self, *exc):
        from paper_2606_12650_gb300 import sem
        sem.autotune_set(*self.key, self.old[0], self.old[1])


def _pair(oracle_mod, nx, ny, nz, N, seed):
    from paper_2606_12650_gb300 import Mesh
    verts = box_vertices(nx, ny, nz, 0.05 if min(nx, ny, nz) > 1 else 0.0, seed=seed)
    return oracle_mod.Problem(nx, ny, nz, N, verts), Mesh(nx, ny, nz, N, verts)


# E = 30 or 105 elements: several blocks and a ragged last block for every epb
@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_f64_ax_parity_every_variant(semlib, oracle_mod, N):
    dims = (3, 2, 5) if N >= 5 else (5, 3, 7)
    P, M = _pair(oracle_mod, *dims, N, seed=10 + N)
    x = normal_field(P.nL, 20 + N)
    y_ref, yg_ref = P.ax_local(x), P.apply(x)
    xd = torch.from_numpy(x).cuda()
    nq2 = (N + 1) ** 2
    epbs = sorted({1, 2, 3, max(1, 256 // nq2), max(1, 512 // nq2)})
    choices = [(COLUMNS, 0)] + [(LINES, e) for e in epbs] + [(LINES_DW, e) for e in epbs]
    for v, epb in choices:
        with variant(F64, N, v, epb):
            yd = torch.full_like(xd, float("nan"))
            M.ax(xd, yd)
            assert _rel(yd.cpu().numpy(), y_ref) < 1e-13, epb
            yg = torch.full_like(xd, float("nan"))
            M.axg(xd, yg)
            assert _rel(yg.cpu().numpy(), yg_ref) < 1e-13, epb
    M.free()


@pytest.mark.parametrize("N,v,epb", [(7, LINES, 1), (7, LINES, 2), (7, LINES, 4), (4, LINES, 3), (8, LINES, 2),
                                     (3, LINES, 8), (7, COLUMNS, 0), (4, COLUMNS, 0), (7, LINES_DW, 1),
                                     (7, LINES_DW, 2), (7, LINES_DW, 4), (4, LINES_DW, 3), (8, LINES_DW, 2),
                                     (3, LINES_DW, 8), (6, LINES_DW, 2)])
def test_cg_history_every_variant(semlib, oracle_mod, N, v, epb):
    P, M = _pair(oracle_mod, 4, 4, 4, N, seed=1)
    b_ref = P.rhs_sin()
    x_ref, it_ref, h_ref = P.cg(b_ref, maxit=100, tol=0.0)
    b = torch.from_numpy(b_ref).cuda()
    x = torch.empty_like(b)
    hist = torch.zeros(101, dtype=torch.float64, device="cuda")
    with variant(F64, N, v, epb):
        it, _ = M.cg_solve(b, x, 0.0, 100, hist)
    assert it == 100 == it_ref
    # rtol 1e-9 while the residual is large; the operators' rounding (~1e-16
    # of ||b||, ~3e-15 in double-word) stays an absolute floor once CG has
    # reduced it by ~1e9 (N <= 4)
    floor = (3e-13 if v == LINES_DW else 1e-14) * h_ref[0]
    np.testing.assert_allclose(hist.cpu().numpy(), h_ref, rtol=1e-9, atol=floor)
    assert _rel(x.cpu().numpy(), x_ref) < 1e-10
    M.free()


@pytest.mark.parametrize("v", [LINES, LINES_DW])
def test_lines_pcg_history(semlib, oracle_mod, v):
    P, M = _pair(oracle_mod, 4, 4, 4, 7, seed=1)
    b_ref = P.rhs_sin()
    x_ref, it_ref, h_ref = P.pcg(b_ref, maxit=60, tol=0.0)
    b = torch.from_numpy(b_ref).cuda()
    x = torch.empty_like(b)
    hist = torch.zeros(61, dtype=torch.float64, device="cuda")
    with variant(F64, 7, v, 2):
        it, _ = M.pcg_solve(b, x, 0.0, 60, hist)
    assert it == 60 == it_ref
    np.testing.assert_allclose(hist.cpu().numpy(), h_ref, rtol=1e-9, atol=0)
    assert _rel(x.cpu().numpy(), x_ref) < 1e-10
    M.free()


@pytest.mark.parametrize("gprec", [0, 1])
@pytest.mark.parametrize("N", [1, 3, 4, 6, 7, 9])
def test_f32_ax_parity_every_variant(semlib, oracle_mod, N, gprec):
    dims = (3, 2, 5) if N >= 5 else (5, 3, 7)
    P, M = _pair(oracle_mod, *dims, N, seed=30 + N)
    x32 = normal_field(P.nL, 60 + N).astype(np.float32)
    Gq = P.G.astype(np.float32).astype(np.float64) if gprec == 0 else bf16_round(P.G)
    y_ref = oracle_mod.ax_local(P.E, N, P.D, Gq, x32.astype(np.float64))
    xd = torch.from_numpy(x32).cuda()
    kind = F32G32 if gprec == 0 else F32G16
    nq2 = (N + 1) ** 2
    epbs = sorted({1, 3, max(1, 256 // nq2), max(1, 512 // nq2)})
    choices = ([(PERSISTENT, 0)] + [(LINES, e) for e in epbs] + [(LINES_ST, e) for e in epbs]
               + [(LINES_PF, e) for e in epbs if gprec == 1])
    for v, epb in choices:
        with variant(kind, N, v, epb):
            yd = torch.full_like(xd, float("nan"))
            M.ax32(xd, yd, gprec)
            assert _rel(yd.cpu().numpy().astype(np.float64), y_ref) < 5e-5, epb
    M.free()


@pytest.mark.parametrize("gprec", [0, 1])
def test_lines_cg_mixed(semlib, oracle_mod, gprec):
    P, M = _pair(oracle_mod, 4, 4, 4, 7, seed=3)
    b_ref = P.mask(P.gs(normal_field(P.nL, 3)))
    it_tol = P.cg(b_ref, maxit=50000, tol=1e-8)[1]
    b = torch.from_numpy(b_ref).cuda()
    x = torch.empty_like(b)
    with variant(F32G32 if gprec == 0 else F32G16, 7, LINES, 4):
        inner, outer, res = M.cg_mixed(b, x, 1e-8, 50, 1e-3, 100000, gprec)
    assert res <= 1e-8
    assert P.true_residual(b_ref, x.cpu().numpy()) <= 1.5e-8
    assert inner <= 1.6 * it_tol + 20
    M.free()


def test_variant_change_recaptures_graphs(semlib, oracle_mod):
    """A solve after a variant change runs the new variant: its history is
    bit-identical to a fresh problem solved with that variant only."""
    P, M = _pair(oracle_mod, 4, 4, 4, 7, seed=1)
    _, M2 = _pair(oracle_mod, 4, 4, 4, 7, seed=1)
    b = torch.from_numpy(P.rhs_sin()).cuda()
    x = torch.empty_like(b)
    h_cols = torch.zeros(81, dtype=torch.float64, device="cuda")
    h_after = torch.zeros_like(h_cols)
    h_fresh = torch.zeros_like(h_cols)
    with variant(F64, 7, COLUMNS):
        M.cg_solve(b, x, 0.0, 80, h_cols)            # captures a graph with the column kernel
    with variant(F64, 7, LINES, 2):
        M.cg_solve(b, x, 0.0, 80, h_after)
        M2.cg_solve(b, x, 0.0, 80, h_fresh)
    assert torch.equal(h_after, h_fresh)
    np.testing.assert_allclose(h_after.cpu().numpy(), h_cols.cpu().numpy(), rtol=1e-9)
    M.free()
    M2.free()


def test_autotune_keeps_fastest_and_round_trips(semlib, oracle_mod, tmp_path):
    from paper_2606_12650_gb300 import Mesh, sem
    M = Mesh(8, 8, 8, 7, box_vertices(8, 8, 8, 0.05, seed=2))
    saved = {k: sem.autotune_get(k, 7) for k in (F64, F32G32, F32G16)}
    try:
        for kind in (F64, F32G16, F32G32):
            cands = M.autotune(kind, reps=3)
            assert len(cands) >= 3
            assert cands[0][0] == (COLUMNS if kind == F64 else PERSISTENT)
            allowed = {F64: (LINES, LINES_DW), F32G32: (LINES, LINES_ST), F32G16: (LINES, LINES_ST, LINES_PF)}[kind]
            assert all(c[0] in allowed and c[1] >= 1 for c in cands[1:])
            assert all(c[2] > 0 for c in cands)
            best = min(cands, key=lambda c: c[2])
            v, e, us = sem.autotune_get(kind, 7)
            assert (v, e) == best[:2] and us == pytest.approx(best[2])
        table = {k: sem.autotune_get(k, 7) for k in (F64, F32G32, F32G16)}
        path = tmp_path / "table.txt"
        sem.autotune_save(str(path))
        assert path.read_text().startswith("#")
        sem.autotune_set(F64, 7, LINES, 1)
        sem.autotune_set(F32G16, 7, PERSISTENT)
        with pytest.raises(sem.SemError):        # the prefetching line kernel is for BF16 factors only
            sem.autotune_set(F32G32, 7, LINES_PF, 4)
        with pytest.raises(sem.SemError):        # staged factors are for FP32 arithmetic only
            sem.autotune_set(F64, 7, LINES_ST, 4)
        with pytest.raises(sem.SemError):        # double-word arithmetic is the FP64 operator's
            sem.autotune_set(F32G32, 7, LINES_DW, 4)
        sem.autotune_load(str(path))
        for k in (F64, F32G32, F32G16):
            v, e, us = sem.autotune_get(k, 7)
            assert (v, e) == table[k][:2] and us == pytest.approx(table[k][2], abs=1e-3)
        # the tuned operator still solves correctly
        P = oracle_mod.Problem(8, 8, 8, 7, box_vertices(8, 8, 8, 0.05, seed=2))
        b_ref = P.mask(P.gs(normal_field(P.nL, 5)))
        b = torch.from_numpy(b_ref).cuda()
        x = torch.empty_like(b)
        it, rel = M.cg_solve(b, x, 1e-9, 10000)
        assert rel <= 1e-9 and P.true_residual(b_ref, x.cpu().numpy()) <= 1.5e-9
        bad = tmp_path / "bad.txt"
        bad.write_text("0 7 2 0\n")     # the persistent kernel has no FP64 form
        with pytest.raises(sem.SemError) as e:
            sem.autotune_load(str(bad))
        assert e.value.code == sem.SEM_EARG
        with pytest.raises(sem.SemError) as e:
            sem.autotune_set(F64, 7, LINES, 0)
        assert e.value.code == sem.SEM_EARG
        with pytest.raises(sem.SemError) as e:
            M.autotune(7)
        assert e.value.code == sem.SEM_EARG
    finally:
        for k, (v, e, _) in saved.items():
            sem.autotune_set(k, 7, v, e)
        M.free()
