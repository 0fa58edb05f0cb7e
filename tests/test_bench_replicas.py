"""The multi-GPU form of the benchmark is N independent replicas (one
network per GPU, no data-path collective).  Its only exchange is the
whole-job reduction of the timing line: the slowest rank's time and the sum
of all ranks' synaptic events.  Checked here on CPU with two gloo ranks."""
import os
import socket
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1), torch.device("cpu"))
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_two_replicas_reduce_max_time_and_total_events():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        assert res[rank] == (15.0, 3000.0)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 777, torch.device("cpu")) == (12.5, 777.0)
