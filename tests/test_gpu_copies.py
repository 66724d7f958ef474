"""Every copy of a global node holds the same bits.

The fused CG update sums the copies of w of each global node in ascending
local index in every element that holds one, so all copies of r -- and
through p = r + beta p and x += alpha p, of p and x -- stay bit-identical
without a separate gather-scatter of the iterates.  Checked on the returned
solution after a fixed number of iterations (no tolerance stop) for the FP64
operator designs, Jacobi PCG and mixed-precision refinement, on a jittered
box whose every face, edge and corner class occurs (3 x 4 x 5 elements).
The copies are grouped by the oracle's global ids.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F64 = 0
COLUMNS, LINES = 0, 1


def _assert_copies_identical(x, gid):
    order = np.argsort(gid, kind="stable")
    g = gid[order]
    bits = np.ascontiguousarray(x[order]).view(np.int64)
    same_node = g[1:] == g[:-1]
    assert same_node.any()
    bad = np.flatnonzero(same_node & (bits[1:] != bits[:-1]))
    assert bad.size == 0, f"{bad.size} copies differ, first at global id {g[bad[0]]}"


@pytest.fixture(scope="module")
def box(semlib, oracle_mod):
    from paper_2606_12650_gb300 import Mesh
    nx, ny, nz, N = 3, 4, 5, 7
    verts = box_vertices(nx, ny, nz, 0.05, seed=9)
    gid, onbdry = oracle_mod.gid(nx, ny, nz, N)
    P = oracle_mod.Problem(nx, ny, nz, N, verts)
    b = P.mask(P.gs(normal_field(P.nL, 11)))
    M = Mesh(nx, ny, nz, N, verts)
    yield M, gid, onbdry, b
    M.free()


@pytest.mark.parametrize("v,epb", [(LINES, 1), (LINES, 3), (COLUMNS, 0)])
def test_cg_iterates_continuous(box, v, epb):
    from paper_2606_12650_gb300 import sem
    M, gid, onbdry, b_np = box
    old = sem.autotune_get(F64, 7)
    sem.autotune_set(F64, 7, v, epb)
    try:
        b = torch.from_numpy(b_np).cuda()
        x = torch.empty_like(b)
        it, _ = M.cg_solve(b, x, 0.0, 37)
        torch.cuda.synchronize()
    finally:
        sem.autotune_set(F64, 7, old[0], old[1])
    assert it == 37
    xh = x.cpu().numpy()
    _assert_copies_identical(xh, gid)
    assert np.all(xh[onbdry != 0] == 0.0)


def test_pcg_iterates_continuous(box):
    M, gid, onbdry, b_np = box
    b = torch.from_numpy(b_np).cuda()
    x = torch.empty_like(b)
    it, _ = M.pcg_solve(b, x, 0.0, 29)
    torch.cuda.synchronize()
    assert it == 29
    xh = x.cpu().numpy()
    _assert_copies_identical(xh, gid)
    assert np.all(xh[onbdry != 0] == 0.0)


@pytest.mark.parametrize("gprec", [0, 1])
def test_mixed_iterates_continuous(box, gprec):
    M, gid, onbdry, b_np = box
    b = torch.from_numpy(b_np).cuda()
    x = torch.empty_like(b)
    M.cg_mixed(b, x, 1e-10, 50, 1e-3, 100000, gprec)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    _assert_copies_identical(xh, gid)
    assert np.all(xh[onbdry != 0] == 0.0)
