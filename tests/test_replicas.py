"""The multi-GPU form is replicas only (HOQRI on one tensor has no exchange step
here): every rank runs its own workload and the job reports the units of all
ranks over the slowest rank's time.  The host logic runs as two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [100.0, 250.0][rank]  # rank 1 is the slow one
    value, ms_max = bench.replica_throughput(ms, 1_000_000, world, "cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_job_throughput_over_slowest_rank():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
        res = dict(out)
    for rank in (0, 1):
        value, ms_max = res[rank]
        assert ms_max == 250.0
        assert abs(value - 2 * 1_000_000 / 0.25) < 1e-6


def test_single_rank_is_plain_throughput():
    import bench
    value, ms_max = bench.replica_throughput(200.0, 500, 1)
    assert ms_max == 200.0 and abs(value - 2500.0) < 1e-9
