"""One problem split by element layers across ranks (processes).

Nekbone runs its CG under MPI with the elements divided among the ranks
(Section VIII-A); the paper names multi-node runs as the next step for its
runtime (Section IX).  Here rank r of W holds the element layers
``slab_ranges(nz, W)[r]`` of an nx x ny x nz box as a libsem "dist" problem;
libsem does all arithmetic (operator, local and interface sums, mask, CG
recurrences) and calls back for the two collective operations, which this
module implements with ``torch.distributed`` on host buffers:

* ``allreduce_sum`` -- the two scalar reductions of each CG iteration;
* ``exchange`` -- the partial sums of the interface plane(s) with the rank
  below and above.

Only argument marshalling lives here; PyTorch supplies the process group.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import sem

ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)
EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double), ctypes.c_int64)


class SemComm(ctypes.Structure):
    """The C struct sem_comm of include/sem.h."""
    _fields_ = [("allreduce_sum", ALLREDUCE_FN), ("exchange", EXCHANGE_FN), ("ctx", ctypes.c_void_p)]


def slab_ranges(nz: int, world: int) -> list[tuple[int, int]]:
    """Element layers [z0, z1) of each rank: contiguous, sizes differing by at
    most one, lower ranks first; every rank gets at least one layer."""
    if world < 1 or nz < world:
        raise ValueError("need at least one element layer per rank")
    base, extra = divmod(nz, world)
    out, z = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def slab_vertices(verts, nx: int, ny: int, z0: int, z1: int) -> np.ndarray:
    """Rows of the global vertex array on the vertex planes z0..z1."""
    plane = (nx + 1) * (ny + 1)
    return np.ascontiguousarray(np.asarray(verts, dtype=np.float64)[z0 * plane:(z1 + 1) * plane])


class TorchComm:
    """sem_comm callbacks on a torch.distributed process group of ranks in z
    order.  Host buffers travel as CPU tensors (gloo) or through the rank's
    GPU (nccl).  A callback that raises returns 1, which libsem reports as
    SEM_ECOMM."""

    def __init__(self, dist, group=None, device=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.device = device if dist.get_backend(group) == "nccl" else None
        self.error = None
        self._ar = ALLREDUCE_FN(self._allreduce)
        self._ex = EXCHANGE_FN(self._exchange)
        self.struct = SemComm(self._ar, self._ex, None)

    def _t(self, arr):
        import torch
        t = torch.from_numpy(arr)
        return t.to(self.device) if self.device is not None else t

    def _allreduce(self, ctx, vals, n):
        try:
            a = np.ctypeslib.as_array(vals, shape=(n,))
            t = self._t(a.copy())
            self.dist.all_reduce(t, group=self.group)
            a[:] = t.cpu().numpy()
            return 0
        except Exception as e:  # reported through SEM_ECOMM
            self.error = e
            return 1

    def _exchange(self, ctx, send_lo, recv_lo, send_hi, recv_hi, n):
        try:
            reqs, outs = [], []
            for peer, snd, rcv in ((self.rank - 1, send_lo, recv_lo), (self.rank + 1, send_hi, recv_hi)):
                if not snd:
                    continue
                s = self._t(np.ctypeslib.as_array(snd, shape=(n,)).copy())
                r = self._t(np.empty(n, dtype=np.float64))
                reqs.append(self.dist.isend(s, peer, group=self.group))
                reqs.append(self.dist.irecv(r, peer, group=self.group))
                outs.append((rcv, r, s))
            for q in reqs:
                q.wait()
            for rcv, r, _ in outs:
                np.ctypeslib.as_array(rcv, shape=(n,))[:] = r.cpu().numpy()
            return 0
        except Exception as e:  # reported through SEM_ECOMM
            self.error = e
            return 1

    def arg(self):
        return sem.HostPtr(ctypes.addressof(self.struct))


class DistMesh:
    """This rank's slab of the nx x ny x nz box (global vertex array
    ``verts``), order N, as a libsem "dist" problem (one sem.run call per
    method)."""

    def __init__(self, nx, ny, nz, N, verts, comm: TorchComm):
        import torch
        self.nx, self.ny, self.nz, self.N = int(nx), int(ny), int(nz), int(N)
        self.comm = comm
        self.z0, self.z1 = slab_ranges(self.nz, comm.world)[comm.rank]
        v = torch.from_numpy(slab_vertices(verts, self.nx, self.ny, self.z0, self.z1)).cuda()
        nb = (1 if comm.rank > 0 else 0) | (2 if comm.rank < comm.world - 1 else 0)
        h = sem.OutInt()
        sem.run("dist_mesh", self.nx, self.ny, self.z1 - self.z0, self.N, v, nb, h)
        self.handle = h.value
        n = sem.OutInt()
        sem.run("dist_info", self.handle, n)
        self.nL = n.value
        npe = (self.N + 1) ** 3
        # this slab's local nodes in the global local-node order
        self.global_slice = slice(self.z0 * self.nx * self.ny * npe, self.z1 * self.nx * self.ny * npe)

    def ax(self, x, y):
        """y = A_local x on this slab's elements."""
        sem.run("dist_ax", self.handle, x, y)

    def gs(self, u):
        """u <- mask(QQ^T u) of the whole problem."""
        sem.run("dist_gs", self.handle, u, self.comm.arg())

    def dot(self, u, v) -> float:
        o = sem.OutDouble()
        sem.run("dist_dot", self.handle, u, v, self.comm.arg(), o)
        return o.value

    def cg_solve(self, b, x, tol: float, maxit: int, hist=None):
        """CG of the whole problem; b, x hold this slab's local nodes.
        Returns (iterations, recursive relative residual); hist (numpy
        float64[maxit + 1]) receives sqrt(<r_k, r_k>)."""
        it, rel = sem.OutInt(), sem.OutDouble()
        sem.run("dist_cg_solve", self.handle, b, x, float(tol), int(maxit), self.comm.arg(),
                sem.HostArray(hist) if hist is not None else None, it, rel)
        return it.value, rel.value

    def free(self):
        if self.handle:
            sem.run("dist_free", self.handle)
            self.handle = 0
