"""The solve server: continuous batching with HBM-budget admission.

Each served result must reach the tolerance with the oracle's own operator
(true residual within 1.5x of tol); a request served alone and inside a
stream of other requests must give bit-identical solutions (its arithmetic
never mixes with other requests'); a budget that fits one request at a time
must serialise the requests and still serve them all.
"""
import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _requests(count, seed, e_hi=96):
    from paper_2606_12650_gb300.serve import make_requests
    return make_requests(count, seed, e_lo=2, e_hi=e_hi, orders=(3, 5, 7))


@pytest.mark.parametrize("mode", [0, 1])
def test_served_results_reach_tolerance(semlib, oracle_mod, mode):
    from paper_2606_12650_gb300 import Server
    from paper_2606_12650_gb300.serve import run_stream
    reqs = _requests(14, seed=7)
    arr = np.linspace(0.0, 0.05, len(reqs))          # overlapping arrivals
    srv = Server(capacity=64, budget_gb=8.0, mode=mode, tol=1e-8, K=8)
    out = run_stream(srv, reqs, arr, collect_x=True)
    srv.close()
    assert np.all(out["latency_ms"] > 0)
    for k, r in enumerate(reqs):
        P = oracle_mod.Problem(r["nx"], r["ny"], r["nz"], r["N"], r["verts"])
        b = P.mask(P.gs(r["f"]))
        if not np.any(b):
            assert not np.any(out["x"][k])
            continue
        assert P.true_residual(b, out["x"][k]) <= 1.5e-8, k


@pytest.mark.parametrize("mode", [0, 1])
def test_alone_and_in_the_mix_are_identical(semlib, mode):
    from paper_2606_12650_gb300 import Server
    from paper_2606_12650_gb300.serve import run_stream
    reqs = _requests(10, seed=11)
    probe = 4
    srv = Server(capacity=64, budget_gb=8.0, mode=mode, tol=1e-8, K=8)
    mixed = run_stream(srv, reqs, np.linspace(0.0, 0.02, len(reqs)), collect_x=True)
    srv.close()
    srv = Server(capacity=64, budget_gb=8.0, mode=mode, tol=1e-8, K=8)
    alone = run_stream(srv, [reqs[probe]], np.zeros(1), collect_x=True)
    srv.close()
    np.testing.assert_array_equal(alone["x"][0], mixed["x"][probe])
    assert alone["iters"][0] == mixed["iters"][probe]


def test_budget_admits_one_at_a_time(semlib):
    """Equal-size requests and a budget for 1.5 of them: one active at a time."""
    from paper_2606_12650_gb300 import Server
    nx, ny, nz, N = 3, 3, 2, 5
    nL = nx * ny * nz * (N + 1) ** 3
    budget_gb = (nL * (48 + 8 + 32 + 8 + 8 + 12 + 16) + 1.2e6) * 1.5 / 1e9
    srv = Server(capacity=64, budget_gb=budget_gb, mode=1, tol=1e-8, K=8)
    t0 = srv.now()
    for k in range(5):
        srv.submit(nx, ny, nz, N, box_vertices(nx, ny, nz, 0.05, seed=k), normal_field(nL, 50 + k), t0,
                   assemble=True)
    done = []
    for _ in range(100000):
        q, a, c = srv.step()
        assert a <= 1
        for tk in srv.drain():   # a result holds its budget share until fetched
            st, it, res, lat = srv.result(tk)
            assert st == 2 and res <= 1e-8 and it > 0
            done.append(tk)
        if c == 5:
            break
    assert len(done) == 5
    srv.close()


def test_unfetched_results_hold_the_budget(semlib):
    """A finished result stays on the device until it is fetched, so it keeps
    its share of the HBM budget: with room for one request, the second is
    admitted only after the first result has been read."""
    from paper_2606_12650_gb300 import Server
    nx, ny, nz, N = 3, 3, 2, 5
    nL = nx * ny * nz * (N + 1) ** 3
    budget_gb = (nL * (48 + 8 + 32 + 8 + 8 + 12 + 16) + 1.2e6) * 1.5 / 1e9
    srv = Server(capacity=64, budget_gb=budget_gb, mode=1, tol=1e-8, K=8)
    t0 = srv.now()
    for k in range(2):
        srv.submit(nx, ny, nz, N, box_vertices(nx, ny, nz, 0.05, seed=k), normal_field(nL, 60 + k), t0,
                   assemble=True)
    first = []
    for _ in range(100000):
        q, a, c = srv.step()
        first += srv.drain()
        if c == 1:
            break
    assert len(first) == 1
    for _ in range(20):                      # the unread result blocks admission
        q, a, c = srv.step()
        assert (q, a, c) == (1, 0, 1)
    assert srv.result(first[0])[0] == 2
    for _ in range(100000):
        q, a, c = srv.step()
        if c == 2:
            break
    (tk,) = srv.drain()
    assert srv.result(tk)[0] == 2
    srv.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_a_bad_request_fails_alone(semlib, oracle_mod, mode):
    """An inverted element in one request (non-positive Jacobian) fails that
    request with SEM_EMESH; the requests before and after it are served and
    give the same bits as when served alone."""
    from paper_2606_12650_gb300 import Server, sem
    from paper_2606_12650_gb300.serve import run_stream
    reqs = _requests(3, seed=13)
    bad = dict(reqs[1])
    verts = box_vertices(2, 2, 2, 0.0, seed=0)
    verts[13, 0] = 1.2                   # the centre vertex pushed past the x = 1 face
    with pytest.raises(ValueError):      # the oracle rejects this mesh too
        oracle_mod.Problem(2, 2, 2, bad["N"], verts)
    bad.update(nx=2, ny=2, nz=2, verts=verts, nL=8 * (bad["N"] + 1) ** 3)
    bad["f"] = normal_field(bad["nL"], 99)
    stream = [reqs[0], bad, reqs[2]]
    srv = Server(capacity=64, budget_gb=8.0, mode=mode, tol=1e-8, K=8)
    mixed = run_stream(srv, stream, np.zeros(3), collect_x=True)
    srv.close()
    assert list(mixed["state"]) == [2, 3, 2]
    assert mixed["iters"][1] == sem.SEM_EMESH
    for k in (0, 2):
        srv = Server(capacity=64, budget_gb=8.0, mode=mode, tol=1e-8, K=8)
        alone = run_stream(srv, [stream[k]], np.zeros(1), collect_x=True)
        srv.close()
        np.testing.assert_array_equal(alone["x"][0], mixed["x"][k])
        assert alone["iters"][0] == mixed["iters"][k]


def test_server_errors(semlib):
    from paper_2606_12650_gb300 import Server, sem
    with pytest.raises(sem.SemError) as e:
        Server(capacity=0)
    assert e.value.code == sem.SEM_EARG
    srv = Server(capacity=4, budget_gb=0.001, mode=1)
    verts = box_vertices(8, 8, 8, 0.05, seed=1)
    with pytest.raises(sem.SemError) as e:   # larger than the whole budget
        srv.submit(8, 8, 8, 7, verts, np.zeros(512 * 512), 0.0)
    assert e.value.code == sem.SEM_ENOMEM
    with pytest.raises(sem.SemError) as e:
        srv.result(12345)
    assert e.value.code == sem.SEM_EHANDLE
    srv.close()
