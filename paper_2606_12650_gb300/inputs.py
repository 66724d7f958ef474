"""Seeded synthetic inputs for the SEM Poisson workload.

This module is the only code that both the CUDA path and the CPU oracle use.
It draws random numbers and lays out box-mesh vertices; it contains none of the
method's arithmetic (no GLL rule, no geometry, no operator, no gather-scatter).

The paper's workload is itself synthetic: a 3D box of E hexahedral elements of
order N (Section VIII-A), with E swept over powers of two (Section VIII-B).
The recipes below stand in for it:

* ``box_vertices`` -- the (nx+1)(ny+1)(nz+1) vertices of a unit-cube box mesh.
  Every vertex not on the cube boundary gets each coordinate moved by
  U(-jitter, +jitter) times the element size in that direction; boundary
  vertices stay fixed, so the Dirichlet boundary stays on the cube faces.
  Vertex index ``v = a + (nx+1)*(b + (ny+1)*c)``; row ``v`` holds (x, y, z).
* ``normal_field`` -- i.i.d. standard normal values (random right-hand sides,
  random operands for operator parity).
* ``near_cubic`` -- factor an element count into nx*ny*nz as close to a cube
  as possible (the paper's E = 2^k sweep, where exact factors are cubic).
* ``cubic_box`` -- sides of a box of about E elements, all within one of
  E^(1/3) (problem mixes; the actual E is recorded).
* ``batch_specs`` / ``arrival_times`` -- problem mixes for batched and served
  runs (element counts log-uniform, orders from a set, Poisson arrivals).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "box_vertices",
    "normal_field",
    "near_cubic",
    "cubic_box",
    "batch_specs",
    "arrival_times",
]


def box_vertices(nx: int, ny: int, nz: int, jitter: float = 0.05, seed: int = 1,
                 xs=None, ys=None, zs=None) -> np.ndarray:
    """Vertices of an nx x ny x nz box mesh of the unit cube, float64 [nv, 3].

    ``xs``/``ys``/``zs`` optionally give non-uniform axis coordinates (strictly
    increasing, from 0 to 1) for an axis-aligned mesh; jitter must then be 0.
    """
    if min(nx, ny, nz) < 1:
        raise ValueError("box needs at least one element per direction")
    axes = []
    for n, given in ((nx, xs), (ny, ys), (nz, zs)):
        if given is None:
            axes.append(np.linspace(0.0, 1.0, n + 1))
        else:
            a = np.asarray(given, dtype=np.float64)
            if a.shape != (n + 1,) or np.any(np.diff(a) <= 0):
                raise ValueError("axis coordinates must be increasing, length n+1")
            if jitter != 0.0:
                raise ValueError("jitter applies to uniform axes only")
            axes.append(a)
    # v = a + (nx+1)*(b + (ny+1)*c): x index fastest
    cz, cy, cx = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    verts = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).copy()
    if jitter != 0.0:
        rng = np.random.default_rng(seed)
        draws = rng.uniform(-jitter, jitter, size=verts.shape)
        iz, iy, ix = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1),
                                 np.arange(nx + 1), indexing="ij")
        interior = ((ix > 0) & (ix < nx) & (iy > 0) & (iy < ny)
                    & (iz > 0) & (iz < nz)).ravel()
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        verts[interior] += draws[interior] * h
    return np.ascontiguousarray(verts)


def normal_field(n: int, seed: int) -> np.ndarray:
    """n i.i.d. N(0, 1) float64 values from a seeded PCG64 stream."""
    return np.random.default_rng(seed).standard_normal(n)


def near_cubic(E: int) -> tuple[int, int, int]:
    """Factor E into (nx, ny, nz) with nx*ny*nz == E and the sides as equal
    as possible (largest side minimal, then the middle one)."""
    if E < 1:
        raise ValueError("E must be positive")
    best = None
    for nz in range(1, E + 1):
        if E % nz:
            continue
        rest = E // nz
        for ny in range(1, rest + 1):
            if rest % ny:
                continue
            nx = rest // ny
            dims = tuple(sorted((nx, ny, nz), reverse=True))
            if best is None or dims < best:
                best = dims
    return best  # (largest, middle, smallest)


def cubic_box(E: float) -> tuple[int, int, int]:
    """Sides of a box of about E elements with all sides within one of
    E^(1/3) (elements of aspect ratio ~1); the product is the actual E."""
    nx = max(1, int(round(E ** (1.0 / 3.0))))
    ny = max(1, int(round(math.sqrt(E / nx))))
    nz = max(1, int(round(E / (nx * ny))))
    return nx, ny, nz


def batch_specs(count: int, seed: int, e_lo: int = 8, e_hi: int = 4096,
                orders=(3, 5, 7, 9)) -> list[dict]:
    """Problem mix: a target E = exp(U[ln e_lo, ln e_hi]) realised as a
    near-cubic box (``cubic_box``; the actual E = nx ny nz is in the spec), N
    drawn uniformly from ``orders``; each problem also gets its own jitter seed
    and right-hand-side seed."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        target = math.exp(rng.uniform(math.log(e_lo), math.log(e_hi)))
        N = int(orders[rng.integers(len(orders))])
        nx, ny, nz = cubic_box(target)
        out.append({"nx": nx, "ny": ny, "nz": nz, "N": N, "E": nx * ny * nz,
                    "mesh_seed": int(rng.integers(1 << 31)),
                    "rhs_seed": int(rng.integers(1 << 31))})
    return out


def arrival_times(rate: float, count: int, seed: int) -> np.ndarray:
    """Cumulative arrival times (seconds) of a Poisson process of ``rate``."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
