"""The multi-rank host logic of bench.py on CPU: two gloo ranks, as torchrun launches them."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    from paper_1403_4661_gb300 import synth
    dist, r, ws, local = bench._dist()
    assert (r, ws, local) == (rank, world, rank)
    ms = bench._max_over_ranks(10.0 + 5.0 * rank, dist)          # the slowest rank decides
    ms_e2e = bench._max_over_ranks(20.0 - 5.0 * rank, dist)
    rate = bench._whole_job_rate(ws, 64, ms)
    c = synth.decaying_coeffs(8, 2, 1000 + rank)                  # each rank its own inputs
    sums = [None] * world
    dist.all_gather_object(sums, float(np.abs(c).sum()))
    dist.barrier()
    out.put((rank, ms, ms_e2e, rate, sums))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, ms_e2e, rate, sums in res:
        assert ms == 15.0 and ms_e2e == 20.0
        assert rate == pytest.approx(2 * 64 / 0.015)
        assert sums[0] != sums[1]        # the ranks transform different batches


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._dist() == (None, 0, 1, 0) or os.environ.get("WORLD_SIZE", "1") != "1"
    assert bench._max_over_ranks(3.5, None) == 3.5
    assert bench._whole_job_rate(1, 64, 100.0) == pytest.approx(640.0)
