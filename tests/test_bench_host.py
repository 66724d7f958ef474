"""Host-side logic of bench.py that needs no GPU: the all-core oracle timing
(spawned replica processes, capped by free host memory)."""
import importlib
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    # imported by its own name: the spawned replica processes import it again
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    return importlib.import_module("bench")


def test_host_memory_is_read(bench):
    m = bench._host_memory_bytes()
    assert m is None or m > 0


def test_replicas_need_room_for_two_copies(bench, monkeypatch):
    monkeypatch.setattr(bench, "_host_memory_bytes", lambda: 1 << 20)
    a = types.SimpleNamespace(nx=2, N=2)
    assert bench.time_oracle_replicas(a, 1, 1) is None


def test_replicas_time_every_step(bench, monkeypatch, oracle_mod):
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    if cores < 2:
        pytest.skip("one host core")
    monkeypatch.setattr(bench, "_host_memory_bytes", lambda: 1 << 40)
    a = types.SimpleNamespace(nx=2, N=2)
    n, times, host = bench.time_oracle_replicas(a, 3, 2)
    assert n == host == cores
    assert len(times) == 2 and all(t > 0 for t in times)


def test_summary_keeps_every_leg_and_tolerates_missing_ones(bench):
    roof = {"kernel": "k", "bound": "hbm", "frac": 0.5}
    s = bench.summarize(10.0, 500.0, roof, None, None, None, None, None)
    assert s["fp64_gdofs"] == 10.0 and s["fp64_solves_per_s"] == 2.0 and s["operator_bound"] == "hbm"
    mixed = {"value": 80.0, "solves_per_s": 16.0, "speedup_solves_vs_fp64": 8.0, "rel_res_true": 9e-9,
             "roofline": {"frac": 0.8}}
    batched = {"fp64": {"solves_per_s": 100.0}, "mixed_bf16": {"solves_per_s": 300.0}}
    served = {"rates": [{"rate_req_s": 100.0, "p50_ms": 5.0, "p99_ms": 9.0, "solves_per_s": 99.0}],
              "closed_loop": {"solves_per_s": 400.0}}
    vs = {"solves": {"mixed_bf16_tol1e-08": {"err_vs_oracle_inf": 1e-9}}}
    s = bench.summarize(10.0, 500.0, roof, mixed, batched, served, {"ms_per_solve": 300.0}, vs)
    assert s["mixed_speedup_vs_fp64"] == 8.0 and s["batched_solves_per_s"]["mixed"] == 300.0
    assert s["served"][0]["p99_ms"] == 9.0 and s["served_closed_loop_solves_per_s"] == 400.0
    assert s["err_vs_oracle_E64"]["mixed_bf16_tol1e-08"] == 1e-9 and s["pcg_ms_per_solve"] == 300.0
