"""The bench's multi-rank bookkeeping on CPU ranks (gloo, world size 2):
the job's time is the slowest rank's and its rate counts every rank's
lattice (each rank sweeps an independent replica; no data is exchanged)."""
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


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]
    mx = bench.max_over_ranks(ms, dist, device="cpu")
    out[rank] = (mx, bench.job_rate(1000 * 1000, 10, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 20.0
    assert abs(res[0][1] - 1e6 * 10 * 2 / (20.0 * 1e6)) < 1e-12
    import bench
    assert bench.max_over_ranks(7.0) == 7.0
