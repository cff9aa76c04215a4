"""World-size-2 runs of the benchmark's multi-rank host logic on CPU (gloo).

With N > 1 the benchmark runs one replica per GPU (the method shards across
right-hand sides and scatterers with no data-path collective): the ranks meet at
a barrier around the timed region, the job time is the slowest rank's, and the
rate counts the units of every rank.  The reference arm runs on rank 0 only.
These tests run those paths as two gloo processes on 127.0.0.1; no GPU is used.
"""
import argparse
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, ws, port):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)


def _args():
    # the reference arm's process group is gloo, which runs on CPU
    return argparse.Namespace(impl="reference", gpus=2, steps=1, warmup=0,
                              workload="sphere_r2_L5", cpu_rhs=1)


def _rate_worker(rank, ws, port, q):
    try:
        _env(rank, ws, port)
        import bench
        import torch.distributed as dist
        got_ws, got_rank, _ = bench.dist_setup(_args())
        bench.barrier(got_ws)
        # rank r took (1 + r) s for its 100 units: the job took the slowest time
        t, rate = bench.job_rate(got_ws, 100, 1.0 + got_rank, "cpu")
        bench.barrier(got_ws)
        dist.destroy_process_group()
        q.put((got_rank, got_ws, t, rate))
    except Exception as e:  # reported to the parent, which fails the test
        q.put((rank, "error", repr(e), None))


def _reference_worker(rank, ws, port, q):
    try:
        _env(rank, ws, port)
        import bench
        import torch.distributed as dist
        out = io.StringIO()
        if rank == 0:
            # rank 0 joins the group only (its oracle run takes minutes)
            bench.dist_setup(_args())
            res = "joined"
        else:
            with redirect_stdout(out):
                res = bench.run_reference(_args())
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, res, out.getvalue(), None))
    except Exception as e:
        q.put((rank, "error", repr(e), None))


def _run_two(target):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = []
    try:
        for _ in procs:
            res.append(q.get(timeout=180))
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return sorted(res, key=lambda r: r[0])


def test_job_rate_two_ranks():
    res = _run_two(_rate_worker)
    for rank, ws, t, rate in res:
        assert ws == 2, (rank, ws, t)
        assert t == pytest.approx(2.0)           # slowest rank's time
        assert rate == pytest.approx(100.0)      # 2 ranks x 100 units / 2 s


def test_reference_arm_runs_on_rank0_only():
    res = _run_two(_reference_worker)
    assert res[0][1] == "joined", res[0]
    rank, ret, out, _ = res[1]
    assert ret is None and out == "", (ret, out)  # rank 1: no work, no line
