"""The bench's multi-rank host logic on CPU (no GPU): with N replicas each
rank times its own product, the job's time is the slowest rank's (max over
ranks, on a world-size-2 gloo process group here), and the reported value is
N x the work of one rank over that time."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        got = bench.max_over_ranks(ms, dist, "cpu")
        out.put((rank, got, bench.whole_job_tflops(world, 2.0e12, got)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]       # both ranks see the slowest time
    # 2 replicas x 2e12 flops in 15 ms
    assert res[0][2] == pytest.approx(2 * 2.0e12 / 15e-3 / 1e12)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.whole_job_tflops(1, 1.0e12, 10.0) == pytest.approx(100.0)


def test_reference_arm_runs_on_rank_zero_only():
    # under torchrun every other rank leaves at once, without work or output
    import argparse
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, 1, 2) is None
