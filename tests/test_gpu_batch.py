"""Batched solves: many problems of different sizes and orders, per order
one persistent launch per CG phase, the orders' chains in parallel.

Checks: every problem of a mixed batch reaches its tolerance with the
oracle's own operator (true residual within 1.5x of tol, the FP64 slack used
throughout), its CG iteration count matches the oracle's within 2 %, and a
problem's solution is bit-identical whether it is solved alone (batch of one)
or inside a larger batch -- the per-problem reductions do not depend on the
batch composition.  Mixed-precision batches reach the same tolerance with at
most 1.6x the FP64 iteration count.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import batch_specs, box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPECS = [(2, 2, 1, 3), (3, 2, 2, 5), (1, 1, 1, 7), (2, 3, 2, 9), (4, 3, 2, 4), (2, 2, 2, 7), (5, 1, 2, 2),
         (1, 2, 1, 1), (3, 3, 3, 6)]


def _build(oracle_mod, specs, with_oracle=True):
    from paper_2606_12650_gb300 import Mesh
    meshes, probs, bs = [], [], []
    for k, (nx, ny, nz, N) in enumerate(specs):
        verts = box_vertices(nx, ny, nz, 0.05 if min(nx, ny, nz) > 1 else 0.0, seed=100 + k)
        meshes.append(Mesh(nx, ny, nz, N, verts))
        P = oracle_mod.Problem(nx, ny, nz, N, verts) if with_oracle else None
        probs.append(P)
        f = normal_field(meshes[-1].nL, 200 + k)
        bs.append(P.mask(P.gs(f)) if P is not None else None)
    return meshes, probs, bs


def _solve(meshes, b_list, tol, mode):
    from paper_2606_12650_gb300 import Batch
    B = Batch(meshes)
    b_all = torch.from_numpy(np.concatenate(b_list)).cuda()
    x_all = torch.full_like(b_all, float("nan"))
    its, res = B.solve(b_all, x_all, tol, 100000, mode)
    torch.cuda.synchronize()
    x = x_all.cpu().numpy()
    xs = [x[o:o + m.nL] for o, m in zip(B.offsets, meshes)]
    B.free()
    return its, res, xs


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_reaches_tolerance_per_problem(semlib, oracle_mod, mode):
    meshes, probs, bs = _build(oracle_mod, SPECS)
    tol = 1e-9
    its, res, xs = _solve(meshes, bs, tol, mode)
    for k, (P, b, x) in enumerate(zip(probs, bs, xs)):
        if not np.any(b):            # every node on the boundary: nothing to solve
            assert its[k] == 0 and res[k] == 0.0 and not np.any(x)
            continue
        it_ref = P.cg(b, maxit=100000, tol=tol)[1]
        assert np.all(np.isfinite(x)), k
        assert res[k] <= tol, (k, res[k])
        assert P.true_residual(b, x) <= 1.5 * tol, k
        if mode == 0:
            assert abs(its[k] - it_ref) <= max(2, 0.02 * it_ref), (k, its[k], it_ref)
        else:
            assert its[k] <= 1.6 * it_ref + 20, (k, its[k], it_ref)
    for m in meshes:
        m.free()


class _body:
    """Make the batch use the column (or line) operator body for every order
    of the spec list, by setting the per-order tuner table; restore after."""

    def __init__(self, mode, variant):
        self.kind = 0 if mode == 0 else (2 if mode == 1 else 1)
        self.variant = variant

    def __enter__(self):
        from paper_2606_12650_gb300 import sem
        self.old = {N: sem.autotune_get(self.kind, N) for N in range(1, 10)}
        for N in range(1, 10):
            if self.variant == "columns":
                sem.autotune_set(self.kind, N, 0 if self.kind == 0 else 2, 0)
            else:
                sem.autotune_set(self.kind, N, 1, max(1, 256 // (N + 1) ** 2))

    def __exit__(self, *exc):
        from paper_2606_12650_gb300 import sem
        for N, (v, e, _) in self.old.items():
            sem.autotune_set(self.kind, N, v, e)


@pytest.mark.parametrize("body", ["columns", "lines"])
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_body_reaches_tolerance(semlib, oracle_mod, mode, body):
    """Each operator body of the batch engine (column or line) on the
    nine-problem mix: tolerance met per problem, checked with the oracle."""
    meshes, probs, bs = _build(oracle_mod, SPECS)
    with _body(mode, body):
        its, res, xs = _solve(meshes, bs, 1e-9, mode)
    for k, (P, b, x) in enumerate(zip(probs, bs, xs)):
        if not np.any(b):
            continue
        assert res[k] <= 1e-9, (k, res[k])
        assert P.true_residual(b, x) <= 1.5e-9, k
    for m in meshes:
        m.free()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_invariance_alone_vs_in_the_mix(semlib, oracle_mod, mode):
    """Problem 3 alone and inside the nine-problem batch: identical bits."""
    meshes, probs, bs = _build(oracle_mod, SPECS)
    _, _, xs_all = _solve(meshes, bs, 1e-8, mode)
    its1, _, xs_one = _solve([meshes[3]], [bs[3]], 1e-8, mode)
    np.testing.assert_array_equal(xs_one[0], xs_all[3])
    # and a different companion set
    sub = [meshes[3], meshes[0], meshes[8]]
    _, _, xs_sub = _solve(sub, [bs[3], bs[0], bs[8]], 1e-8, mode)
    np.testing.assert_array_equal(xs_sub[0], xs_all[3])
    for m in meshes:
        m.free()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_every_order_alone_and_mixed(semlib, oracle_mod, mode):
    """Two problems of each order N = 1..9 (18 problems, nine per-order
    kernel chains in one round): each reaches its tolerance under the
    oracle's operator, and the first problem of every order gives the same
    bits alone (batch of one) as in the full mix."""
    specs = []
    for N in range(1, 10):
        specs.append((2, 2, 1, N))
        specs.append((3, 2, 2, N) if N <= 6 else (2, 2, 2, N))
    meshes, probs, bs = _build(oracle_mod, specs)
    tol = 1e-9
    its, res, xs = _solve(meshes, bs, tol, mode)
    for k, (P, b, x) in enumerate(zip(probs, bs, xs)):
        if not np.any(b):
            continue
        assert res[k] <= tol, (k, specs[k], res[k])
        assert P.true_residual(b, x) <= 1.5 * tol, (k, specs[k])
    for k in range(0, len(specs), 2):
        its1, res1, xs1 = _solve([meshes[k]], [bs[k]], tol, mode)
        assert its1[0] == its[k], specs[k]
        np.testing.assert_array_equal(xs1[0], xs[k])
    for m in meshes:
        m.free()


def test_batch_of_random_mix(semlib, oracle_mod):
    """32 problems drawn like the batched workload (E log-uniform, N in
    {3,5,7,9}, smaller E range): FP64 and mixed; sampled problems against the
    oracle, the rest by their own true residual."""
    from paper_2606_12650_gb300 import Mesh
    specs = batch_specs(32, seed=4, e_lo=8, e_hi=256)
    meshes, bs = [], []
    for s in specs:
        verts = box_vertices(s["nx"], s["ny"], s["nz"], 0.05 if min(s["nx"], s["ny"], s["nz"]) > 1 else 0.0,
                             seed=s["mesh_seed"])
        m = Mesh(s["nx"], s["ny"], s["nz"], s["N"], verts)
        f = torch.from_numpy(normal_field(m.nL, s["rhs_seed"])).cuda()
        m.gs(f)
        m.mask(f)
        meshes.append(m)
        bs.append(f.cpu().numpy())
    for mode in (0, 1):
        its, res, xs = _solve(meshes, bs, 1e-8, mode)
        assert np.all(res <= 1e-8)
        for k in (0, 7, 19, 31):
            s = specs[k]
            verts = box_vertices(s["nx"], s["ny"], s["nz"],
                                 0.05 if min(s["nx"], s["ny"], s["nz"]) > 1 else 0.0, seed=s["mesh_seed"])
            P = oracle_mod.Problem(s["nx"], s["ny"], s["nz"], s["N"], verts)
            assert P.true_residual(bs[k], xs[k]) <= 1.5e-8
        for k, m in enumerate(meshes):
            xd = torch.from_numpy(xs[k]).cuda()
            bd = torch.from_numpy(bs[k]).cuda()
            assert m.true_res(bd, xd) <= 1.5e-8
    for m in meshes:
        m.free()


def test_batch_errors(semlib, oracle_mod):
    from paper_2606_12650_gb300 import Batch, Mesh, sem
    m = Mesh(2, 2, 2, 3, box_vertices(2, 2, 2, 0.05, seed=1))
    with pytest.raises(sem.SemError) as e:
        Batch([m, m])
    assert e.value.code == sem.SEM_EARG
    B = Batch([m])
    b = torch.zeros(m.nL, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        B.solve(b, torch.empty_like(b), 1e-8, 100, mode=5)
    assert e.value.code == sem.SEM_EARG
    with pytest.raises(sem.SemError) as e:   # a problem held by a batch cannot be freed
        m.free()
    assert e.value.code == sem.SEM_EARG
    its, res = B.solve(b, torch.empty_like(b), 1e-8, 100, mode=0)   # zero rhs: nothing to do
    assert its[0] == 0 and res[0] == 0.0
    B.free()
    m.free()
