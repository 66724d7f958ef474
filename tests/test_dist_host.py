"""One problem split by element layers across ranks: host side, no GPU.

* the slab partition and each slab's vertex rows;
* the sem_comm callbacks of ``dist.TorchComm`` over gloo (world 2 and 3,
  processes on the CPU): the allreduce sums, the exchange delivers the rank
  below's data to recv_lo and the rank above's to recv_hi;
* the decomposition itself, emulated with the oracle on each rank's slab: the
  slab's own direct-stiffness sum, the exchange of the interface-plane partial
  sums (lower rank's partial first), and the mask of the global cube faces
  give the global mask(QQ^T u) restricted to the slab; the slab's weights
  with interface multiplicities doubled are the global 1/multiplicity.  The
  plane maps and the mask here are written from the oracle's lattice ids,
  independently of libsem's (whose kernels the GPU tests check against the
  oracle).
"""
import ctypes
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_ranges_cover_layers_contiguously():
    from paper_2606_12650_gb300.dist import slab_ranges
    for nz in range(1, 12):
        for world in range(1, nz + 1):
            rs = slab_ranges(nz, world)
            assert rs[0][0] == 0 and rs[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            sizes = [z1 - z0 for z0, z1 in rs]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slab_ranges(2, 3)


def test_slab_vertices_are_the_global_planes():
    from paper_2606_12650_gb300.dist import slab_vertices
    from paper_2606_12650_gb300.inputs import box_vertices
    nx, ny, nz = 3, 2, 5
    v = box_vertices(nx, ny, nz, 0.05, seed=3)
    s = slab_vertices(v, nx, ny, 2, 4)
    V = v.reshape(nz + 1, ny + 1, nx + 1, 3)
    np.testing.assert_array_equal(s.reshape(3, ny + 1, nx + 1, 3), V[2:5])


def _plane_maps(gid, lx, ly, lz):
    """Per face (z0, z1): for each plane point, its local copies ascending."""
    gz = gid // (lx * ly)
    out = []
    for face in (0, lz - 1):
        sel = np.nonzero(gz == face)[0]
        pts = gid[sel] % (lx * ly)
        order = np.lexsort((sel, pts))
        out.append((pts[order], sel[order]))
    return out


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import datetime
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        import oracle
        from paper_2606_12650_gb300.dist import TorchComm, slab_ranges, slab_vertices
        from paper_2606_12650_gb300.inputs import box_vertices, normal_field
        comm = TorchComm(dist)
        out = {}
        # -- the callbacks, called as libsem calls them
        vals = (ctypes.c_double * 2)(rank + 1.0, 10.0 * rank)
        assert comm.struct.allreduce_sum(None, vals, 2) == 0
        out["allreduce"] = (vals[0], vals[1])
        n = 3
        has_lo, has_hi = rank > 0, rank < world - 1
        snd_lo = (ctypes.c_double * n)(*[100.0 * rank + k for k in range(n)]) if has_lo else None
        snd_hi = (ctypes.c_double * n)(*[100.0 * rank + 50 + k for k in range(n)]) if has_hi else None
        rcv_lo = (ctypes.c_double * n)() if has_lo else None
        rcv_hi = (ctypes.c_double * n)() if has_hi else None
        cast = lambda a: ctypes.cast(a, ctypes.POINTER(ctypes.c_double)) if a is not None else None
        assert comm.struct.exchange(None, cast(snd_lo), cast(rcv_lo), cast(snd_hi), cast(rcv_hi), n) == 0
        out["recv_lo"] = list(rcv_lo) if has_lo else None
        out["recv_hi"] = list(rcv_hi) if has_hi else None
        # -- the decomposition, emulated with the oracle on this rank's slab
        nx, ny, nz, N = 3, 2, 2 * world, 3
        verts = box_vertices(nx, ny, nz, 0.05, seed=7)
        G = oracle.Problem(nx, ny, nz, N, verts)
        u = normal_field(G.nL, 8)
        ref = G.mask(G.gs(u))
        z0, z1 = slab_ranges(nz, world)[rank]
        npe = (N + 1) ** 3
        sl = slice(z0 * nx * ny * npe, z1 * nx * ny * npe)
        S = oracle.Problem(nx, ny, z1 - z0, N, slab_vertices(verts, nx, ny, z0, z1))
        v = S.gs(u[sl])                                  # the slab's own sum
        lx, ly, lz = nx * N + 1, ny * N + 1, (z1 - z0) * N + 1
        planes = _plane_maps(S.gid, lx, ly, lz)
        for face, has, own_lower in ((0, has_lo, False), (1, has_hi, True)):
            if not has:
                continue
            pts, copies = planes[face]
            first = np.unique(pts, return_index=True)[1]
            part = np.ascontiguousarray(v[copies[first]])   # one value per plane point
            other = np.empty_like(part)
            peer = rank - 1 if face == 0 else rank + 1
            reqs = [dist.isend(torch.from_numpy(part), peer), dist.irecv(torch.from_numpy(other), peer)]
            for rq in reqs:
                rq.wait()
            tot = part + other if own_lower else other + part
            v[copies] = tot[np.searchsorted(np.unique(pts), pts)]
        gx, gy, gz = S.gid % lx, (S.gid // lx) % ly, S.gid // (lx * ly)
        glob_face = (gx == 0) | (gx == lx - 1) | (gy == 0) | (gy == ly - 1) | \
                    ((gz == 0) & (not has_lo)) | ((gz == lz - 1) & (not has_hi))
        v[glob_face] = 0.0
        out["gs_err"] = float(np.abs(v - ref[sl]).max() / np.abs(ref).max())
        iface = ((gz == 0) & has_lo) | ((gz == lz - 1) & has_hi)
        c_glob = 1.0 / (S.mult * np.where(iface, 2.0, 1.0))
        out["c_equal"] = bool(np.array_equal(c_glob, G.c[sl]))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_callbacks_and_decomposition(world, oracle_mod):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tot = (sum(r + 1.0 for r in range(world)), sum(10.0 * r for r in range(world)))
    for r in range(world):
        out = res[r]
        assert out["allreduce"] == tot
        if r > 0:     # from the rank below: its z1 (hi) side
            assert out["recv_lo"] == [100.0 * (r - 1) + 50 + k for k in range(3)]
        if r < world - 1:
            assert out["recv_hi"] == [100.0 * (r + 1) + k for k in range(3)]
        assert out["gs_err"] <= 1e-15
        assert out["c_equal"]
