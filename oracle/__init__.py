"""CPU oracle for the SEM Poisson operator and CG (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_2606_12650_gb300``): the numerics live in ``sem_oracle.c`` (plain C,
FP64, compiled without FMA contraction) and this file only marshals numpy
arrays through ctypes.  The one module both sides use is
``paper_2606_12650_gb300.inputs``, which draws the seeded synthetic inputs and
holds none of the method's arithmetic.

The paper names the Poisson operator ("ax", Section VIII-B), the
gather-scatter kernel (Section V-B, Fig. "gs" transform: outer loop over
global ids, order-enforced inner loops over copies) and the CG solve of
Nekbone without preconditioner (Section VIII-A), but writes out none of the
formulas; ``sem_oracle.c`` spells out the textbook SEM formulation it uses.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsemoracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile sem_oracle.c into a shared library (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # SEM_ORACLE_LIB lets the mutation test load a deliberately broken copy
        override = os.environ.get("SEM_ORACLE_LIB")
        lib = ctypes.CDLL(override if override else build())
        lib.orc_gll.argtypes = [ctypes.c_int, _d, _d]
        lib.orc_gll.restype = ctypes.c_int
        lib.orc_deriv.argtypes = [ctypes.c_int, _d, _d]
        lib.orc_deriv.restype = None
        lib.orc_nodes.argtypes = [ctypes.c_int] * 4 + [_d, _d, _d]
        lib.orc_nodes.restype = None
        lib.orc_nodes_rel.argtypes = [ctypes.c_int] * 4 + [_d, _d, _d]
        lib.orc_nodes_rel.restype = None
        lib.orc_geometry.argtypes = [ctypes.c_long, ctypes.c_int, _d, _d, _d, _d, _d]
        lib.orc_geometry.restype = ctypes.c_long
        lib.orc_ax_local.argtypes = [ctypes.c_long, ctypes.c_int, _d, _d, _d, _d]
        lib.orc_ax_local.restype = None
        lib.orc_gid.argtypes = [ctypes.c_int] * 4 + [_i64, _u8]
        lib.orc_gid.restype = None
        lib.orc_gs.argtypes = [ctypes.c_long, _i64, ctypes.c_long, _d, _d, _u8]
        lib.orc_gs.restype = None
        lib.orc_mask.argtypes = [ctypes.c_long, _u8, _d]
        lib.orc_mask.restype = None
        lib.orc_dot.argtypes = [ctypes.c_long, _d, _d, _d]
        lib.orc_dot.restype = ctypes.c_double
        lib.orc_cg.argtypes = [ctypes.c_long, ctypes.c_int, _d, _d, ctypes.c_long, _i64,
                               ctypes.c_long, _u8, _d, _d, _d, ctypes.c_int,
                               ctypes.c_double, _d]
        lib.orc_cg.restype = ctypes.c_int
        lib.orc_diag.argtypes = [ctypes.c_long, ctypes.c_int, _d, _d, ctypes.c_long, _i64, ctypes.c_long,
                                 _u8, _d]
        lib.orc_diag.restype = None
        lib.orc_pcg.argtypes = [ctypes.c_long, ctypes.c_int, _d, _d, ctypes.c_long, _i64,
                                ctypes.c_long, _u8, _d, _d, _d, _d, ctypes.c_int, ctypes.c_double, _d]
        lib.orc_pcg.restype = ctypes.c_int
        _lib = lib
        return lib


def _p(a, ty=_d):
    return a.ctypes.data_as(ty)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gll(N: int):
    """GLL nodes and weights (ascending), float64 arrays of length N+1."""
    lib = _load()
    xi = np.empty(N + 1)
    w = np.empty(N + 1)
    if lib.orc_gll(N, _p(xi), _p(w)) != 0:
        raise ValueError("GLL needs N >= 1")
    return xi, w


def deriv(N: int, xi=None):
    """Derivative matrix D[i, j] = l_j'(xi_i) on the GLL nodes."""
    lib = _load()
    if xi is None:
        xi, _ = gll(N)
    D = np.empty((N + 1, N + 1))
    lib.orc_deriv(N, _p(_f64(xi)), _p(D))
    return D


def nodes(nx, ny, nz, N, verts, xi=None):
    """Nodal coordinates [nL, 3] of every local node (trilinear element map)."""
    lib = _load()
    if xi is None:
        xi, _ = gll(N)
    E = nx * ny * nz
    X = np.empty((E * (N + 1) ** 3, 3))
    lib.orc_nodes(nx, ny, nz, N, _p(_f64(verts)), _p(_f64(xi)), _p(X))
    return X


def nodes_rel(nx, ny, nz, N, verts, xi=None):
    """Nodal coordinates [nL, 3] relative to each element's first vertex
    (the trilinear map of the vertex differences): the input of ``geometry``
    for a box mesh, free of the O(1) offset's rounding."""
    lib = _load()
    if xi is None:
        xi, _ = gll(N)
    E = nx * ny * nz
    X = np.empty((E * (N + 1) ** 3, 3))
    lib.orc_nodes_rel(nx, ny, nz, N, _p(_f64(verts)), _p(_f64(xi)), _p(X))
    return X


def geometry(E, N, X, D, w):
    """Geometric factors G [nL, 6] = (rr, rs, rt, ss, st, tt) and mass B [nL]."""
    lib = _load()
    nL = E * (N + 1) ** 3
    G = np.empty((nL, 6))
    B = np.empty(nL)
    rc = lib.orc_geometry(E, N, _p(_f64(X)), _p(_f64(D)), _p(_f64(w)), _p(G), _p(B))
    if rc != 0:
        raise ValueError(f"non-positive Jacobian at local node {-rc - 1}")
    return G, B


def ax_local(E, N, D, G, u):
    """Unassembled local Poisson action y_e = A_e u_e for every element."""
    lib = _load()
    u = _f64(u)
    y = np.empty_like(u)
    lib.orc_ax_local(E, N, _p(_f64(D)), _p(_f64(G)), _p(u), _p(y))
    return y


def gid(nx, ny, nz, N):
    """Global id of every local node and its cube-boundary flag."""
    lib = _load()
    nL = nx * ny * nz * (N + 1) ** 3
    g = np.empty(nL, dtype=np.int64)
    b = np.empty(nL, dtype=np.uint8)
    lib.orc_gid(nx, ny, nz, N, _p(g, _i64), _p(b, _u8))
    return g, b


def weighted_dot(c, u, v):
    """sum_l c_l u_l v_l in ascending l (FP64); c=None means unit weights."""
    lib = _load()
    u = _f64(u)
    c = np.ones_like(u) if c is None else _f64(c)
    return lib.orc_dot(u.size, _p(c), _p(u), _p(_f64(v)))


class Problem:
    """One box-mesh Poisson problem, every quantity computed by the oracle.

    Attributes: xi, w, D, X (nodal coordinates), G, B, gid, onbdry, nG,
    mult (copies per global id, per local node), c = 1/mult.
    """

    def __init__(self, nx, ny, nz, N, verts):
        self.nx, self.ny, self.nz, self.N = int(nx), int(ny), int(nz), int(N)
        self.E = self.nx * self.ny * self.nz
        self.n = self.N + 1
        self.np_ = self.n ** 3
        self.nL = self.E * self.np_
        self.verts = _f64(verts)
        self.xi, self.w = gll(self.N)
        self.D = deriv(self.N, self.xi)
        self.X = nodes(self.nx, self.ny, self.nz, self.N, self.verts, self.xi)
        # J from coordinates relative to each element's first vertex (same
        # derivative; rounding relative to the element size)
        Xrel = nodes_rel(self.nx, self.ny, self.nz, self.N, self.verts, self.xi)
        self.G, self.B = geometry(self.E, self.N, Xrel, self.D, self.w)
        del Xrel
        self.gid, self.onbdry = gid(self.nx, self.ny, self.nz, self.N)
        self.nG = (self.nx * self.N + 1) * (self.ny * self.N + 1) * (self.nz * self.N + 1)
        counts = np.bincount(self.gid, minlength=self.nG)
        self.mult = counts[self.gid].astype(np.float64)
        self.c = 1.0 / self.mult

    # -- operators ----------------------------------------------------------
    def ax_local(self, u):
        return ax_local(self.E, self.N, self.D, self.G, u)

    def gs(self, u):
        """QQ^T u (copies summed in ascending local index), returns a new array."""
        lib = _load()
        v = np.array(u, dtype=np.float64, copy=True)
        s = np.empty(self.nG)
        seen = np.empty(self.nG, dtype=np.uint8)
        lib.orc_gs(self.nL, _p(self.gid, _i64), self.nG, _p(v), _p(s), _p(seen, _u8))
        return v

    def mask(self, u):
        lib = _load()
        v = np.array(u, dtype=np.float64, copy=True)
        lib.orc_mask(self.nL, _p(self.onbdry, _u8), _p(v))
        return v

    def apply(self, u):
        """Assembled, masked operator mask(QQ^T(A_local u))."""
        return self.mask(self.gs(self.ax_local(u)))

    def dot(self, u, v):
        lib = _load()
        return lib.orc_dot(self.nL, _p(self.c), _p(_f64(u)), _p(_f64(v)))

    # -- right-hand sides ----------------------------------------------------
    def rhs_from_source(self, f):
        """b = mask(QQ^T(B * f)) for nodal source values f."""
        return self.mask(self.gs(self.B * _f64(f)))

    def rhs_sin(self):
        """Manufactured u = sin(pi x) sin(pi y) sin(pi z): f = 3 pi^2 u."""
        x, y, z = self.X[:, 0], self.X[:, 1], self.X[:, 2]
        f = 3.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
        return self.rhs_from_source(f)

    def rhs_random(self, seed):
        """Assembled random right-hand side: b = mask(QQ^T(f)), f ~ N(0,1) per local node."""
        from paper_2606_12650_gb300.inputs import normal_field
        return self.mask(self.gs(normal_field(self.nL, seed)))

    # -- solver --------------------------------------------------------------
    def cg(self, b, maxit=100, tol=0.0):
        """Unpreconditioned CG from x0 = 0.  Returns (x, iters, hist) with
        hist[k] = sqrt(<r_k, r_k>_c)."""
        lib = _load()
        b = _f64(b)
        x = np.empty_like(b)
        hist = np.zeros(maxit + 1)
        it = lib.orc_cg(self.E, self.N, _p(self.D), _p(self.G), self.nL,
                        _p(self.gid, _i64), self.nG, _p(self.onbdry, _u8), _p(self.c),
                        _p(b), _p(x), int(maxit), float(tol), _p(hist))
        return x, it, hist[: it + 1].copy()

    def diag(self):
        """Diagonal of the assembled, masked operator (zero on masked nodes)."""
        lib = _load()
        d = np.empty(self.nL)
        lib.orc_diag(self.E, self.N, _p(self.D), _p(self.G), self.nL, _p(self.gid, _i64), self.nG,
                     _p(self.onbdry, _u8), _p(d))
        return d

    def pcg(self, b, maxit=100, tol=0.0, dinv=None):
        """Jacobi-preconditioned CG from x0 = 0; hist[k] = ||r_k||_c.
        Returns (x, iters, hist)."""
        lib = _load()
        if dinv is None:
            d = self.diag()
            dinv = np.where(d > 0.0, 1.0 / np.where(d > 0.0, d, 1.0), 0.0)
        b = _f64(b)
        x = np.empty_like(b)
        hist = np.zeros(maxit + 1)
        it = lib.orc_pcg(self.E, self.N, _p(self.D), _p(self.G), self.nL, _p(self.gid, _i64), self.nG,
                         _p(self.onbdry, _u8), _p(self.c), _p(_f64(dinv)), _p(b), _p(x), int(maxit),
                         float(tol), _p(hist))
        return x, it, hist[: it + 1].copy()

    def true_residual(self, b, x):
        """||b - A x||_c / ||b||_c in FP64."""
        r = _f64(b) - self.apply(x)
        return np.sqrt(self.dot(r, r) / self.dot(b, b))


if __name__ == "__main__":  # pragma: no cover - manual build helper
    print(build(force="--force" in sys.argv))
