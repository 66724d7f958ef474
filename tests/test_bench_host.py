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
