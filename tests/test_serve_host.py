"""The serving load driver (serve.run_stream, serve.sweep) on the host, no
GPU: a scripted stand-in for the server checks the driver's bookkeeping --
every request submitted at its arrival time, each finished ticket mapped back
to its request, the state / iterations / residual / latency the server
reports passed through unchanged, the span from the first arrival to the
last completion, the throughput and the latency percentiles of a sweep row.
"""
import time

import numpy as np
import pytest

from paper_2606_12650_gb300 import serve


class FakeServer:
    """Completes each request a fixed number of steps after it was submitted;
    a request whose N is 0 fails (state 3).  Latency = completion - arrival on
    the same clock the driver reads."""

    def __init__(self, service_steps=3, **_):
        self.t0 = time.monotonic()
        self.service_steps = service_steps
        self.pending = {}      # ticket -> [steps left, arrival, request N]
        self.done = {}         # ticket -> (state, iters, res, latency_ms)
        self.finished = []
        self.next_ticket = 1
        self.submitted = []    # (ticket, arrival_s, submit time)
        self.closed = False

    def now(self):
        return time.monotonic() - self.t0

    def submit(self, nx, ny, nz, N, verts, f, arrival_s, assemble=False):
        tk = self.next_ticket
        self.next_ticket += 1
        self.pending[tk] = [self.service_steps, arrival_s, N]
        self.submitted.append((tk, arrival_s, self.now()))
        return tk

    def step(self):
        for tk in list(self.pending):
            left, arrival, N = self.pending[tk]
            if left > 1:
                self.pending[tk][0] = left - 1
                continue
            del self.pending[tk]
            lat = 1e3 * (self.now() - arrival)
            self.done[tk] = (3, -6, float("nan"), lat) if N == 0 else (2, 10 * tk, 1e-9 * tk, lat)
            self.finished.append(tk)
        return 0, len(self.pending), len(self.done)

    def drain(self):
        out, self.finished = self.finished, []
        return out

    def result(self, tk, x=None):
        st, it, res, lat = self.done.pop(tk)
        if x is not None and st == 2:
            x[:] = tk
        return st, it, res, lat

    def close(self):
        self.closed = True


def _requests(n, bad=()):
    return [dict(nx=1, ny=1, nz=1, N=0 if k in bad else 3, verts=None, f=None, nL=4) for k in range(n)]


def test_run_stream_maps_tickets_and_passes_results_through():
    srv = FakeServer(service_steps=2)
    reqs = _requests(12, bad={5})
    arrivals = np.linspace(0.0, 0.03, 12)
    out = serve.run_stream(srv, reqs, arrivals, collect_x=True)
    assert len(srv.submitted) == 12
    for tk, arrival, t_sub in srv.submitted:    # never submitted before its arrival time
        assert t_sub >= arrival - 1e-6
    # request k got ticket k + 1 (submitted in arrival order)
    for k in range(12):
        tk = k + 1
        if k == 5:
            assert out["state"][k] == 3 and out["iters"][k] == -6 and np.isnan(out["rel_res"][k])
        else:
            assert out["state"][k] == 2 and out["iters"][k] == 10 * tk
            assert out["rel_res"][k] == pytest.approx(1e-9 * tk)
            np.testing.assert_array_equal(out["x"][k], np.full(4, float(tk)))
    assert np.all(out["latency_ms"] > 0)
    ends = arrivals + out["latency_ms"] / 1e3
    assert out["span_s"] == pytest.approx(ends.max() - arrivals[0])
    assert out["mean_depth"] >= 0


def test_sweep_row_statistics(monkeypatch):
    made = []

    def fake_server(**kw):
        srv = FakeServer(service_steps=1)
        made.append(srv)
        return srv

    monkeypatch.setattr(serve, "Server", fake_server)
    monkeypatch.setattr(serve, "make_requests", lambda count, seed: _requests(count))
    rows = serve.sweep([2000.0, 4000.0], 40, seed=3, K=16)
    assert len(rows) == 2 and all(s.closed for s in made)
    for row, rate in zip(rows, (2000.0, 4000.0)):
        assert row["rate_req_s"] == rate and row["requests"] == 40
        assert 0 < row["p50_ms"] <= row["p99_ms"]
        assert row["mean_ms"] > 0
        assert row["solves_per_s"] > 0
