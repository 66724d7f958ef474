"""Problem sizes beyond a fixed reduction buffer.

A problem's grid-sum buffer is sized from its element count, so a CG
operator launch of one element per block works for any E.  E = 52^3 =
140608 at N = 1 with one element per block is above the 131072 block slots
that smaller problems get: the operator (DFMA lines and double-word) matches
the oracle within 1e-13 and the first 5 CG residuals match the oracle's
within rtol 1e-9.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NX, N = 52, 1


@pytest.mark.parametrize("variant", [1, 5], ids=["lines", "double_word"])
def test_more_blocks_than_the_default_slots(semlib, oracle_mod, variant):
    from paper_2606_12650_gb300 import Mesh, sem
    verts = box_vertices(NX, NX, NX, 0.05, seed=8)
    P = oracle_mod.Problem(NX, NX, NX, N, verts)
    assert P.E > 131072
    M = Mesh(NX, NX, NX, N, verts)
    saved = sem.autotune_get(0, N)
    try:
        sem.autotune_set(0, N, variant, 1)          # one element per block: E blocks
        x = normal_field(P.nL, 9)
        xd = torch.from_numpy(x).cuda()
        yd = torch.full_like(xd, float("nan"))
        M.ax(xd, yd)
        y_ref = P.ax_local(x)
        assert np.abs(yd.cpu().numpy() - y_ref).max() / np.abs(y_ref).max() < 1e-13
        b_ref = P.mask(P.gs(normal_field(P.nL, 10)))
        _, it_ref, h_ref = P.cg(b_ref, maxit=5, tol=0.0)
        b = torch.from_numpy(b_ref).cuda()
        xs = torch.empty_like(b)
        hist = torch.zeros(6, dtype=torch.float64, device="cuda")
        it, _ = M.cg_solve(b, xs, 0.0, 5, hist)
        assert it == 5 == it_ref
        np.testing.assert_allclose(hist.cpu().numpy(), h_ref, rtol=1e-9, atol=0)
    finally:
        sem.autotune_set(0, N, saved[0], saved[1])
        M.free()
