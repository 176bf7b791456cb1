"""The N-rank path of bench.py on the CPU: two gloo ranks (world size 2) run
the bench's whole-job aggregation.  Each rank steps its own replica (no
data-path collective), so the only cross-rank steps are the barrier and the
maximum of the timed durations; the whole-job rate is the units of all ranks
over the slowest rank's time.  Also the environment parsing that torchrun
feeds."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, rate = bench.job_rate(10.0 + 5.0 * rank, 1e9, dist)
    dist.barrier()
    out.put((rank, ms, rate))
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, rate in res:
        assert ms == 15.0
        assert rate == pytest.approx(2e9 / 0.015, rel=1e-12)


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.job_rate(20.0, 5e8)
    assert ms == 20.0 and rate == pytest.approx(2.5e10)


def test_dist_env_reads_torchrun_variables(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("WORLD_SIZE", "4")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.dist_env() == (3, 4, 1)
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(v)
    assert bench.dist_env() == (0, 1, 0)
