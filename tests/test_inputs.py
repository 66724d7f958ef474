"""The seeded input generators shared by the CUDA path and the oracle: the
properties the readings of the paper rely on (boundary vertices fixed, jitter
bounded by the stated fraction of the element size, exact factorisations,
problem mixes within their ranges, Poisson arrivals), and reproducibility."""
import math

import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import (arrival_times, batch_specs, box_vertices, cubic_box,
                                           near_cubic, normal_field)


@pytest.mark.parametrize("dims", [(1, 1, 1), (3, 4, 5), (8, 2, 1)])
def test_box_vertices_boundary_fixed_interior_bounded(dims):
    nx, ny, nz = dims
    jit = 0.05
    v = box_vertices(nx, ny, nz, jit, seed=7)
    ref = box_vertices(nx, ny, nz, 0.0)
    assert v.shape == ((nx + 1) * (ny + 1) * (nz + 1), 3)
    c, b, a = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    a, b, c = a.ravel(), b.ravel(), c.ravel()
    # vertex index a + (nx+1)(b + (ny+1)c), x fastest, on the uniform grid
    np.testing.assert_allclose(ref, np.stack([a / nx, b / ny, c / nz], axis=1), rtol=0, atol=1e-15)
    interior = (a > 0) & (a < nx) & (b > 0) & (b < ny) & (c > 0) & (c < nz)
    np.testing.assert_array_equal(v[~interior], ref[~interior])
    h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
    d = np.abs(v - ref) / h
    assert np.all(d <= jit * (1 + 1e-12))
    if interior.any():
        assert d[interior].max() > 0.5 * jit   # the jitter is actually applied


def test_box_vertices_seeded_and_axes():
    a = box_vertices(4, 4, 4, 0.05, seed=3)
    np.testing.assert_array_equal(a, box_vertices(4, 4, 4, 0.05, seed=3))
    assert not np.array_equal(a, box_vertices(4, 4, 4, 0.05, seed=4))
    xs = [0.0, 0.2, 0.7, 1.0]
    v = box_vertices(3, 1, 1, 0.0, xs=xs)
    np.testing.assert_array_equal(v[:4, 0], xs)
    with pytest.raises(ValueError):
        box_vertices(3, 1, 1, 0.05, xs=xs)
    with pytest.raises(ValueError):
        box_vertices(3, 1, 1, 0.0, xs=[0.0, 0.5, 0.5, 1.0])
    with pytest.raises(ValueError):
        box_vertices(0, 1, 1)


def test_normal_field_seeded_standard_normal():
    f = normal_field(1 << 16, 11)
    np.testing.assert_array_equal(f, normal_field(1 << 16, 11))
    assert abs(f.mean()) < 0.02 and abs(f.std() - 1.0) < 0.02


@pytest.mark.parametrize("E", [1, 2, 7, 12, 64, 96, 2 ** 13, 2 ** 14, 97])
def test_near_cubic_exact_and_balanced(E):
    nx, ny, nz = near_cubic(E)
    assert nx * ny * nz == E and nx >= ny >= nz >= 1
    # no exact factorisation has a smaller largest side (then middle side)
    for c in range(1, E + 1):
        if E % c:
            continue
        for b in range(1, E // c + 1):
            if (E // c) % b == 0:
                assert tuple(sorted((E // c // b, b, c), reverse=True)) >= (nx, ny, nz)


@pytest.mark.parametrize("E", [8, 100, 1000, 4096, 5000.5, 8192])
def test_cubic_box_sides_near_cube_root(E):
    s = cubic_box(E)
    r = E ** (1.0 / 3.0)
    assert all(abs(d - r) <= 1.0 + 1e-9 or d == 1 for d in s)
    assert abs(math.prod(s) / E - 1.0) < 0.5


def test_batch_specs_ranges_and_seeds():
    specs = batch_specs(256, seed=4, e_lo=8, e_hi=4096, orders=(3, 5, 7, 9))
    assert len(specs) == 256
    assert {s["N"] for s in specs} == {3, 5, 7, 9}
    for s in specs:
        assert s["E"] == s["nx"] * s["ny"] * s["nz"]
        assert 4 <= s["E"] <= 2 * 4096
    assert len({s["mesh_seed"] for s in specs}) == 256
    assert specs == batch_specs(256, seed=4, e_lo=8, e_hi=4096, orders=(3, 5, 7, 9))
    # log-uniform targets: about half of the problems below the geometric mean
    below = sum(s["E"] < math.sqrt(8 * 4096) for s in specs)
    assert 90 < below < 166


def test_arrival_times_poisson():
    t = arrival_times(200.0, 20000, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.03      # mean inter-arrival 1/rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential: cv = 1
    np.testing.assert_array_equal(t, arrival_times(200.0, 20000, seed=5))
