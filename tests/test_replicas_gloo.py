"""The N-GPU bench path (replicas only: independent problems, a barrier and
the max of the per-rank timings) with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(world, backend="gloo")
    assert (r, w) == (rank, world)
    bench.barrier(w)
    # each rank reports its own time; the job time is the slowest rank's
    mx = bench.max_over_ranks(10.0 + 5.0 * rank, w)
    with open(os.path.join(outdir, "rank%d" % rank), "w") as f:
        f.write(repr(mx))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    vals = [float(open(tmp_path / ("rank%d" % r)).read()) for r in range(world)]
    assert vals == [15.0, 15.0]


def test_replica_throughput_counts_every_rank():
    import bench
    # 1M cells x 40 steps per rank, slowest rank 50 ms, 4 ranks
    assert bench.replica_value(1 << 20, 50.0, 1) == pytest.approx((1 << 20) / 0.05)
    assert bench.replica_value(40 * (1 << 20), 50.0, 4) == pytest.approx(4 * 40 * (1 << 20) / 0.05)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    bench.reference_arm(argparse.Namespace(steps=1, warmup=3, gpus=2))
    assert capsys.readouterr().out == ""
