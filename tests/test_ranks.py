"""Replica runs on several ranks, host side only (gloo, two processes on the
CPU): the job's time is the slowest rank's, its work the sum over ranks;
ranks draw disjoint problems; the reference arm prints from rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    from paper_2606_12650_gb300.inputs import batch_specs
    from paper_2606_12650_gb300.ranks import Job, rank_env, rank_seed
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, local, w = rank_env()
        job = Job(w, dist, device="cpu", local=local)
        job.barrier()
        t, units = job.aggregate(10.0 + 3.0 * r, 100.0 * (r + 1))
        rate, t_max, u_sum = job.throughput(2.0 - r, 5.0)
        specs = batch_specs(4, seed=rank_seed(4, r), e_lo=8, e_hi=64)
        gathered = [None] * w
        dist.all_gather_object(gathered, [(s["mesh_seed"], s["rhs_seed"]) for s in specs])
        job.barrier()
        out.put((r, t, units, rate, t_max, u_sum, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_figures():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, t, units, rate, t_max, u_sum, gathered in res:
        assert t == 13.0 and units == 300.0            # max over ranks, sum over ranks
        assert t_max == 2.0 and u_sum == 10.0 and rate == 5.0
        seeds0, seeds1 = (set(map(tuple, g)) for g in gathered)
        assert not seeds0 & seeds1                       # no problem is solved twice


def test_single_rank_job_is_identity():
    from paper_2606_12650_gb300.ranks import Job
    job = Job(1)
    job.barrier()
    assert job.aggregate(4.5, 7) == (4.5, 7.0)
    assert job.throughput(2.0, 8.0) == (4.0, 2.0, 8.0)


def test_reference_arm_prints_on_rank_zero_only():
    """A non-zero rank of `bench.py --impl reference` exits 0 without work or
    output (the oracle is timed on rank 0 alone)."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_line_on_rank_zero(oracle_mod):
    """Rank 0 of the reference arm prints one JSON line with the contract's
    keys; a small problem keeps it quick."""
    env = dict(os.environ, RANK="0", LOCAL_RANK="0", WORLD_SIZE="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--nx", "4",
                        "--N", "3", "--steps", "2", "--warmup", "1", "--cpu-iters", "3"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "GDOF/s" and line["value"] > 0
    for k in ("metric", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
    cb = line["cpu_baseline"]
    # one oracle process per host core that fits in memory, or the single-threaded oracle
    assert cb["cores"] >= 1 and cb["value"] == line["value"]
    assert ("independent processes" in cb["sample"]) == (cb["cores"] > 1)
