"""The N > 1 bench path on CPU: two gloo ranks, each with its own system;
the whole-job throughput uses the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, seconds, out):
    import torch.distributed as dist

    from paper_2405_04808_gb300 import replicas as R
    from paper_2405_04808_gb300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = R.rank_seed(1000, rank)
        prob = W.vdp(n=16, seed=seed)
        dist.barrier()
        value = R.job_throughput(seconds[rank], units_per_rank=5, world=world)
        out[rank] = (value, seed, float(prob.b[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    seconds = [2.0, 4.0]
    mp.spawn(_worker, args=(world, port, seconds, out), nprocs=world, join=True)
    v0, s0, b0 = out[0]
    v1, s1, b1 = out[1]
    assert v0 == v1 == pytest.approx(world * 5 / 4.0)   # 10 solves in the slowest rank's 4 s
    assert s0 != s1 and b0 != b1                          # ranks solve different systems


def test_single_rank_needs_no_process_group():
    from paper_2405_04808_gb300 import replicas as R
    assert R.job_throughput(0.5, 3, 1) == pytest.approx(6.0)
    with pytest.raises(ValueError):
        R.job_throughput(0.0, 3, 1)
