"""The multi-process path of bench.py on CPU (gloo, world size 2): every rank
runs its own replica of the index on its own query batch (no data-path
collective), and the job's time is the slowest rank's, shared by an
all-reduce MAX."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 7.5 * rank
    out[rank] = bench.max_over_ranks(local_ms, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: 17.5, 1: 17.5}


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
