"""The multi-GPU form of the benchmark: independent replicas, one process per GPU, with the
slowest replica's time for the whole job (the path does not shard; there is no data-path
collective).  The host logic runs here as world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import bench
    r, w, local = bench.dist_env()
    dev = torch.device("cpu")
    bench.init_dist(w, dev)
    bench.barrier(w)
    ms = 10.0 + 5.0 * r                       # rank 1 is the slow replica
    ms_max = bench.max_over_ranks(ms, w, dev)
    units = 2.0e12                            # per replica
    rate = bench.whole_job_rate(units, w, ms_max * 1e-3)
    out.put((r, w, local, ms_max, rate))
    dist.destroy_process_group()


def test_replicas_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, ms_max, rate) in enumerate(res):
        assert (rank, w, local) == (r, world, r)
        assert ms_max == 15.0                          # the max over ranks, on every rank
        assert rate == pytest.approx(world * 2.0e12 / 15e-3)


def _reference_rank(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import contextlib
    import io

    import bench
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        if rank != 0:
            bench.run_reference(bench.argparse.Namespace(steps=1, warmup=0))
    out.put((rank, buf.getvalue()))


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun the oracle arm runs on rank 0 alone; the other ranks print nothing."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_reference_rank, args=(1, world, port, q))
    p.start()
    rank, text = q.get(timeout=120)
    p.join(timeout=60)
    assert p.exitcode == 0 and rank == 1 and text == ""
