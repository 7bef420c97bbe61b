"""Host logic of the multi-rank benchmark on CPU (gloo, two ranks): each
rank times its own replica; the job's time is the slowest rank's and the
rate counts every rank's sites."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = [0.5, 2.0][rank]
    t = bench.rank_max(local_seconds, dist, device="cpu")
    out[rank] = (t, bench.job_rate(world, 1000.0, 10, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        res = dict(out)
    assert res[0][0] == 2.0 and res[1][0] == 2.0
    # 2 ranks x 1000 sites x 10 steps in 2 s
    assert res[0][1] == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.rank_max(1.25) == 1.25
    assert bench.job_rate(1, 2e6, 5, 0.5) == pytest.approx(20.0)
