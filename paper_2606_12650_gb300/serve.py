"""Open-loop load driver for the solve server.

Requests arrive at the times of a Poisson process; the driver submits each
one at its arrival time (open loop: arrivals do not wait for completions),
steps the server, and collects finished tickets.  Everything on the device is
done by libsem's server (admission, continuous batching, retirement); this
module only keeps time and computes latency statistics.
"""
from __future__ import annotations

import time

import numpy as np

from .inputs import arrival_times, batch_specs, box_vertices, normal_field
from .mesh import Server


def make_requests(count: int, seed: int, e_lo: int = 8, e_hi: int = 8192, orders=(5, 7)) -> list[dict]:
    """Request mix: near-cubic boxes of log-uniform element count, N from
    ``orders``, jittered vertices, nodal source f ~ N(0, 1)."""
    out = []
    for s in batch_specs(count, seed=seed, e_lo=e_lo, e_hi=e_hi, orders=orders):
        jit = 0.05 if min(s["nx"], s["ny"], s["nz"]) > 1 else 0.0
        verts = box_vertices(s["nx"], s["ny"], s["nz"], jit, seed=s["mesh_seed"])
        nL = s["E"] * (s["N"] + 1) ** 3
        out.append(dict(s, verts=verts, f=normal_field(nL, s["rhs_seed"]), nL=nL))
    return out


def run_stream(server: Server, requests: list[dict], arrivals, collect_x: bool = False) -> dict:
    """Submit requests at their arrival times (seconds from now), serve them
    all, and return per-request latency, iterations and residuals (state 2:
    solved; 3: failed, iterations then hold the error code)."""
    n = len(requests)
    t0 = server.now()
    tick_of, done, xs = {}, {}, {}
    i = 0
    depth = []
    while len(done) < n:
        now = server.now() - t0
        while i < n and arrivals[i] <= now:
            r = requests[i]
            tk = server.submit(r["nx"], r["ny"], r["nz"], r["N"], r["verts"], r["f"], t0 + float(arrivals[i]),
                               assemble=True)
            tick_of[tk] = i
            i += 1
        queued, active, _ = server.step()
        depth.append(queued + active)
        for tk in server.drain():
            k = tick_of[tk]
            x = np.empty(requests[k]["nL"]) if collect_x else None
            st, it, res, lat = server.result(tk, x)
            done[k] = (lat, it, res, st)
            if collect_x:
                xs[k] = x
        if queued == 0 and active == 0 and i < n:
            time.sleep(max(0.0, float(arrivals[i]) - (server.now() - t0)))
    lat = np.array([done[k][0] for k in range(n)])
    first = float(arrivals[0]) if n else 0.0
    last_done = max(float(arrivals[k]) + lat[k] / 1e3 for k in range(n)) if n else 0.0
    return {"latency_ms": lat, "iters": np.array([done[k][1] for k in range(n)]),
            "rel_res": np.array([done[k][2] for k in range(n)]), "x": xs,
            "state": np.array([done[k][3] for k in range(n)]),
            "span_s": last_done - first, "mean_depth": float(np.mean(depth)) if depth else 0.0}


def sweep(rates, count: int, seed: int, mode: int = 1, budget_gb: float = 40.0, capacity: int = 512,
          K: int = 16, tol: float = 1e-8) -> list[dict]:
    """p50 / p99 latency and throughput for each arrival rate (req/s)."""
    rows = []
    for q, rate in enumerate(rates):
        reqs = make_requests(count, seed + q)
        arr = arrival_times(rate, count, seed + 100 + q) - 0.0
        srv = Server(capacity=capacity, budget_gb=budget_gb, mode=mode, tol=tol, K=K)
        try:
            out = run_stream(srv, reqs, arr)
        finally:
            srv.close()
        lat = out["latency_ms"]
        rows.append({"rate_req_s": rate, "requests": count, "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                     "solves_per_s": count / out["span_s"] if out["span_s"] > 0 else None,
                     "mean_queue_depth": out["mean_depth"], "max_rel_res": float(out["rel_res"].max())})
    return rows
