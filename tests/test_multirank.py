"""The benchmark's N > 1 path (independent replicas, one per rank) on CPU:
world_size 2 under gloo.  Each rank times its own replica; the job's time is
the slowest rank's (max over ranks, seen by every rank) and the job's
throughput counts every rank's cell-updates."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 31.0][rank]
    got = bench.max_over_ranks(local_ms, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "r%d" % rank), "w") as f:
        f.write(repr(got))


def test_max_over_ranks_gloo_world2(tmp_path):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = [float(open(os.path.join(tmp_path, "r%d" % r)).read()) for r in range(2)]
    assert got == [31.0, 31.0]


def test_job_value_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, 1, "cpu") == 7.0
    one = bench.job_value(1, 8192 * 8192, 100, 10, 250.0)
    assert one == pytest.approx(8192 * 8192 * 100 * 10 / 0.25 / 1e9)
    # weak scaling: N replicas in the slowest rank's time
    assert bench.job_value(4, 8192 * 8192, 100, 10, 250.0) == pytest.approx(4 * one)
