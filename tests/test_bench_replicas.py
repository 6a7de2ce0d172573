"""The multi-GPU path of bench.py is independent replicas: a barrier, the slowest
rank's timed duration (all_reduce MAX) and whole-job throughput. Checked with two
gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = [120.0, 150.0][rank]
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, bench.job_throughput(300, world, ms), bench.replica_seed(1000, rank))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 150.0
    assert out[0][1] == pytest.approx(2 * 300 / 0.150)
    assert out[0][2] != out[1][2]


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_throughput(100, 1, 50.0) == pytest.approx(2000.0)


def test_all_cores_oracle_pool_sums_concurrent_loops():
    """The all-cores CPU baseline: independent single-thread oracle loops of the small
    workload in fresh processes, their rates summed."""
    import bench
    r = bench.run_oracle_pool("scao_8m_64px", 0.5, 3, 2)
    assert r["processes"] == 2 and r["steps"] >= 2 and r["value"] > 0
