"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank reports its own step time; every rank must see the slowest one, and the whole-job
rate must count the units of both ranks over it.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    from paper_0910_0992_gb300.replicas import Replicas

    reps = Replicas("gloo")
    reps.barrier()
    ms = 10.0 * (rank + 1)
    slowest = reps.max(ms)
    rate = reps.whole_job_rate(100.0, slowest * 1e-3)
    out[rank] = (reps.rank, reps.world, slowest, rate)
    reps.barrier()
    reps.close()


def test_two_gloo_ranks_share_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in range(world):
        r, w, slowest, rate = out[rank]
        assert (r, w) == (rank, world)
        assert slowest == 20.0
        assert rate == pytest.approx(2 * 100.0 / 0.020)


def test_single_rank_is_a_no_op(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_0910_0992_gb300.replicas import Replicas

    reps = Replicas("gloo")
    assert (reps.world, reps.rank) == (1, 0)
    assert reps.max(3.5) == 3.5
    assert reps.whole_job_rate(10.0, 2.0) == 5.0
    reps.close()
