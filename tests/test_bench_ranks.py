"""The multi-rank arithmetic of bench.py, on two CPU ranks over gloo: every
rank learns the slowest rank's time, the whole-job value counts the units of
all ranks over that time (weak scaling: one replica of the workload per
rank), and the reference arm runs on rank 0 only."""
import argparse
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        ms = bench.slowest_rank(dist, 10.0 + 5.0 * rank, "cpu")  # rank 1 is the slower one
        value = bench.job_throughput(1000, ws, ms / 1000.0)
        dist.barrier()
        out.put((rank, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_every_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
    assert [p.exitcode for p in procs] == [0, 0]
    assert [r for r, _, _ in res] == [0, 1]
    assert res[0][1] == res[1][1] == 15.0
    assert res[0][2] == res[1][2] == pytest.approx(1000 * 2 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.slowest_rank(None, 12.5, "cpu") == 12.5
    assert bench.job_throughput(10, 1, 2.0) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    args = argparse.Namespace(log2n=20, workload="rgg", warmup=3, steps=5, coarsener="lp", initial="bfs",
                              lp_relax="0/1", reb_objective="cut")
    # a non-zero rank returns at once: no workload generated, no oracle run
    assert bench.run_reference(args, 2, 1) == 0
