"""``Mesh``: one box-mesh Poisson problem held by libsem, addressed by handle.

Each method is one ``sem.run`` call (argument marshalling only).  Vectors are
CUDA tensors of float64 on local nodes (``nL = E (N+1)^3`` entries, layout
``l = i + n(j + n(k + n e))``), or host arrays mirrored with ``sem.update``.
"""
from __future__ import annotations

import numpy as np

from . import sem


class Mesh:
    def __init__(self, nx: int, ny: int, nz: int, N: int, verts):
        self.nx, self.ny, self.nz, self.N = int(nx), int(ny), int(nz), int(N)
        h = sem.OutInt()
        if isinstance(verts, np.ndarray):
            v = np.ascontiguousarray(verts, dtype=np.float64)
            sem.update(v, sem.SEM_TO)
            try:
                sem.run("mesh", self.nx, self.ny, self.nz, self.N, v, h)
            finally:
                sem.update(v, sem.SEM_FREE)
        else:
            sem.run("mesh", self.nx, self.ny, self.nz, self.N, verts, h)
        self.handle = h.value
        i = [sem.OutInt() for _ in range(4)]
        sem.run("info", self.handle, *i)
        self.nL, self.nG, self.n_shared, self.n_masked = (o.value for o in i)
        self.E = self.nx * self.ny * self.nz

    # operators -------------------------------------------------------------
    def ax(self, x, y):
        sem.run("ax", self.handle, x, y)

    def axg(self, x, y):
        sem.run("axg", self.handle, x, y)

    def gs(self, u):
        sem.run("gs", self.handle, u)

    def mask(self, u):
        sem.run("mask", self.handle, u)

    def dot(self, u, v) -> float:
        o = sem.OutDouble()
        sem.run("dot", self.handle, u, v, o)
        return o.value

    # set-up products -------------------------------------------------------
    def geom(self, G, B):
        sem.run("geom", self.handle, G, B)

    def nodes(self, X):
        sem.run("nodes", self.handle, X)

    def gs_map(self, ptr, idx):
        sem.run("gs_map", self.handle, ptr, idx)

    def rhs(self, f, b):
        sem.run("rhs", self.handle, f, b)

    def rhs_sin(self, b):
        sem.run("rhs_sin", self.handle, b)

    # solver ----------------------------------------------------------------
    def cg_solve(self, b, x, tol: float, maxit: int, hist=None):
        it, res = sem.OutInt(), sem.OutDouble()
        sem.run("cg_solve", self.handle, b, x, float(tol), int(maxit), it, res, hist)
        return it.value, res.value

    def ax32(self, x, y, gprec: int = 1):
        """y = A_local x in FP32 with G stored FP32 (gprec 0) or BF16 (gprec 1)."""
        sem.run("ax32", self.handle, x, y, int(gprec))

    def cg_mixed(self, b, x, tol: float, max_outer: int = 50, inner_tol: float = 1e-3,
                 inner_maxit: int = 100000, gprec: int = 1, hist_outer=None):
        """Mixed-precision iterative refinement; returns (inner_iters, outer_iters,
        true relative residual)."""
        i, o, r = sem.OutInt(), sem.OutInt(), sem.OutDouble()
        sem.run("cg_mixed", self.handle, b, x, float(tol), int(max_outer), float(inner_tol),
                int(inner_maxit), int(gprec), i, o, r, hist_outer)
        return i.value, o.value, r.value

    def pcg_solve(self, b, x, tol: float, maxit: int, hist=None):
        """Jacobi-preconditioned CG; returns (iters, ||r||_c / ||b||_c)."""
        it, res = sem.OutInt(), sem.OutDouble()
        sem.run("pcg_solve", self.handle, b, x, float(tol), int(maxit), it, res, hist)
        return it.value, res.value

    def jacobi(self, dinv):
        sem.run("jacobi", self.handle, dinv)

    def autotune(self, kind: int, reps: int = 10):
        """Tune the operator variant for this problem's order (sem.autotune)."""
        return sem.autotune(self.handle, kind, reps)

    def true_res(self, b, x) -> float:
        o = sem.OutDouble()
        sem.run("true_res", self.handle, b, x, o)
        return o.value

    def free(self):
        if self.handle:
            sem.run("mesh_free", self.handle)
            self.handle = 0


class Batch:
    """Problems solved together: per order present, each CG phase is one
    persistent launch over that order's problems (sem.h, "batch_solve")."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        hs = np.array([m.handle for m in self.meshes], dtype=np.int64)
        h = sem.OutInt()
        sem.run("batch", len(hs), sem.HostArray(hs), h)
        self.handle = h.value
        n, tot = sem.OutInt(), sem.OutInt()
        sem.run("batch_info", self.handle, n, tot)
        self.n, self.nL_total = n.value, tot.value
        self.offsets = np.concatenate([[0], np.cumsum([m.nL for m in self.meshes])])[:-1]

    def solve(self, b_all, x_all, tol: float, maxit: int = 100000, mode: int = 0,
              inner_tol: float = 1e-3, max_outer: int = 50):
        """Returns (iters per problem, relative residual per problem)."""
        its = np.zeros(self.n, dtype=np.int64)
        res = np.zeros(self.n, dtype=np.float64)
        tot, mx = sem.OutInt(), sem.OutDouble()
        sem.run("batch_solve", self.handle, b_all, x_all, float(tol), int(maxit), int(mode),
                float(inner_tol), int(max_outer), tot, mx, sem.HostArray(its), sem.HostArray(res))
        return its, res

    def free(self):
        if self.handle:
            sem.run("batch_free", self.handle)
            self.handle = 0


class Server:
    """Continuous-batching solve server (one sem.run call per method)."""

    def __init__(self, capacity: int = 256, budget_gb: float = 40.0, mode: int = 1, tol: float = 1e-8,
                 inner_tol: float = 1e-3, K: int = 16, maxit: int = 100000):
        h = sem.OutInt()
        sem.run("serve_open", int(capacity), float(budget_gb), int(mode), float(tol), float(inner_tol),
                int(K), int(maxit), h)
        self.handle = h.value

    def now(self) -> float:
        o = sem.OutDouble()
        sem.run("serve_now", self.handle, o)
        return o.value

    def submit(self, nx, ny, nz, N, verts, b, arrival: float, assemble: bool = False) -> int:
        """Queue a request; with assemble=True, b is a nodal source f and the
        server solves with mask(QQ^T f)."""
        t = sem.OutInt()
        v = np.ascontiguousarray(verts, dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        sem.run("serve_submit", self.handle, int(nx), int(ny), int(nz), int(N), sem.HostArray(v),
                sem.HostArray(bb), int(bool(assemble)), float(arrival), t)
        return t.value

    def drain(self, cap: int = 4096):
        """Tickets completed since the last drain."""
        out = np.zeros(cap, dtype=np.int64)
        n = sem.OutInt()
        sem.run("serve_drain", self.handle, sem.HostArray(out), int(cap), n)
        return out[: n.value].tolist()

    def step(self):
        """Returns (queued, active, completed)."""
        q, a, c = sem.OutInt(), sem.OutInt(), sem.OutInt()
        sem.run("serve_step", self.handle, q, a, c)
        return q.value, a.value, c.value

    def result(self, ticket: int, x=None):
        """Returns (state, iters, rel_res, latency_ms); x (host numpy array or
        CUDA tensor) receives the solution when state == 2."""
        st, it, res, lat = sem.OutInt(), sem.OutInt(), sem.OutDouble(), sem.OutDouble()
        xa = sem.HostArray(x) if isinstance(x, np.ndarray) else x
        sem.run("serve_result", self.handle, int(ticket), xa, st, it, res, lat)
        return st.value, it.value, res.value, lat.value

    def close(self):
        if self.handle:
            sem.run("serve_close", self.handle)
            self.handle = 0
