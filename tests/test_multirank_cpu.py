"""Multi-process (N > 1) host logic of bench.py, run as two gloo ranks on CPU.

Every rank builds an independent problem (weak scaling, no data-path
collective): the ranks' windows must differ, the step time is the maximum
over ranks, the value counts the units of all ranks, and the reference arm
prints from rank 0 only.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        bench.LMAX = 40
        Wt, Wc, Wp = bench.windows_for_rank(r)
        sums = [None] * world
        dist.all_gather_object(sums, float(Wt.sum() + Wc.sum() + Wp.sum()))
        slowest = bench.max_over_ranks(1.0 + 0.5 * r, w, "cpu")
        value = bench.job_value(w, 1000.0, slowest)
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.ragged_seed0(r))

        class A:
            steps, warmup, gpus = 1, 0, world
        buf = io.StringIO()
        if r != 0:
            with redirect_stdout(buf):
                bench.run_reference(A, r, w)   # rank 0 alone works and prints
        dist.barrier()
        out_q.put((r, sums, slowest, value, seeds, buf.getvalue()))
    finally:
        if dist.is_initialized():
            dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, sums, slowest, value, seeds, printed = q.get(timeout=240)
        res[r] = (sums, slowest, value, seeds, printed)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        sums, slowest, value, seeds, printed = res[r]
        assert sums[0] != sums[1]                 # independent problems per rank
        assert slowest == 1.5                     # max over ranks
        assert np.isclose(value, 2 * 1000.0 / 1.5)  # all ranks' units / the slowest time
        assert seeds[0] != seeds[1]
    assert res[1][4] == ""                        # the reference arm prints on rank 0 only
