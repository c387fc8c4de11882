"""The multi-rank path of bench.py on CPU: two ranks over the gloo backend (127.0.0.1).

The benchmark shards independent sweeps over ranks (rank r solves the sweep with data seed 1 + r;
no collective on the data path) and reduces only the timing: every timed region is the maximum
over ranks (bench.max_over_all_ranks), and the whole-job value counts the units of all ranks.
Under the reference arm only rank 0 runs and prints; the other ranks return without work.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_1502_04070_gb300 import workloads
        local_ms = [12.5, 40.25][rank]                  # rank 1 is the slow one
        m = bench.max_over_all_ranks(local_ms, "cpu")
        fn, gn = workloads.random_nodal(3, 1 + rank)    # the sweep's data seed of this rank
        td.barrier()
        out.put((rank, m, float(fn.sum()), float(gn.sum())))
    finally:
        td.destroy_process_group()


def test_two_ranks_reduce_the_timing_by_max_and_shard_the_data():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, m, fs, gs = out.get(timeout=120)
        res[r] = (m, fs, gs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 40.25
    assert res[0][1:] != res[1][1:]                     # different data on the two ranks


def test_max_over_ranks_without_a_process_group_is_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_all_ranks(3.5, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(None, rank=1, world=2) is None
    assert buf.getvalue() == ""


def test_whole_job_value_counts_every_rank():
    """value = solves per step x unknowns per solve x steps x ranks / max time (weak scaling)."""
    sys.path.insert(0, ROOT)
    import bench
    n = bench.dofs(bench.K_LEVEL)
    assert n == 2356227                                 # h = 1/512: 2 x 1023^2 + 513^2 unknowns
    units = len(bench.BETAS) * n
    one = bench.job_throughput(units, 3, 1, 80.0)
    assert np.isclose(one, units * 3 / 0.080)
    assert np.isclose(bench.job_throughput(units, 3, 2, 80.0), 2 * one)
