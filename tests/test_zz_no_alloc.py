"""The allocation-free dot product (sem_dot_noalloc) against the CPU oracle
and the regular "dot" entry point.

sem_dot_noalloc exists for callers that cannot let a library allocate device
memory (graph capture that forbids allocation, allocation-free real-time
loops, device memory owned by another framework).  Its scratch is a static
device array shared by every call, so each test calls it twice in a row on
different data and checks every result against the oracle's weighted dot of
host copies and against the regular entry point, with the dot-product
tolerance used by the parity tests: |d - d_ref| <= 1e-13 sqrt(<u,u><v,v>).
The file is named to run last.
"""
import math

import numpy as np
import pytest

from paper_2606_12650_gb300.inputs import box_vertices, normal_field

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_dot_noalloc_matches_oracle_and_dot_on_two_calls(semlib, oracle_mod):
    from paper_2606_12650_gb300 import Mesh, sem
    M = Mesh(8, 8, 8, 7, box_vertices(8, 8, 8, 0.05, seed=4))   # nL = 262144: 128 blocks
    mult = torch.ones(M.nL, dtype=torch.float64, device="cuda")
    M.gs(mult)                                                  # QQ^T 1 = multiplicity
    c = (1.0 / mult).contiguous()
    c_host = c.cpu().numpy()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        u_h = normal_field(M.nL, 50 + 2 * call)
        v_h = normal_field(M.nL, 51 + 2 * call)
        u = torch.from_numpy(u_h).cuda()
        v = torch.from_numpy(v_h).cuda()
        ref = oracle_mod.weighted_dot(c_host, u_h, v_h)
        scale = math.sqrt(oracle_mod.weighted_dot(c_host, u_h, u_h) * oracle_mod.weighted_dot(c_host, v_h, v_h))
        sem.dot_noalloc(c, u, v, M.nL, out[call:call + 1], sem.stream().cuda_stream)
        torch.cuda.synchronize()
        got = float(out[call].item())
        assert abs(got - ref) <= 1e-13 * scale, (call, got, ref)
        assert abs(got - M.dot(u, v)) <= 1e-13 * scale, (call, got)
    M.free()


@pytest.mark.parametrize("n", [1, 2047, 2049, 1000003])
def test_dot_noalloc_unit_weights_ragged(semlib, oracle_mod, n):
    """c = NULL (unit weights) with n > 0, including sizes that leave the last
    block of 2048 entries partly filled, twice in a row."""
    from paper_2606_12650_gb300 import sem
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        u_h = normal_field(n, 70 + 2 * call)
        v_h = normal_field(n, 71 + 2 * call)
        u = torch.from_numpy(u_h).cuda()
        v = torch.from_numpy(v_h).cuda()
        sem.dot_noalloc(None, u, v, n, out, sem.stream().cuda_stream)
        torch.cuda.synchronize()
        got = float(out.item())
        ref = oracle_mod.weighted_dot(None, u_h, v_h)
        scale = math.sqrt(float(np.dot(u_h, u_h)) * float(np.dot(v_h, v_h)))
        assert abs(got - ref) <= 1e-13 * scale, (n, call, got, ref)


def test_dot_noalloc_limits(semlib):
    from paper_2606_12650_gb300 import sem
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:
        sem.dot_noalloc(None, x, x, 16777217, out, sem.stream().cuda_stream)
    assert e.value.code == sem.SEM_ERANGE
    sem.dot_noalloc(None, x, x, 0, out, sem.stream().cuda_stream)   # empty sum
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
