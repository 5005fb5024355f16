"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): the
path shards as independent replicas (no data-path collective), so what
crosses ranks is the timing: each timed region's step time is the slowest
rank's, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench._dist()
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, dist, "cpu")  # rank 1 is the slow one
        single = bench.max_over_ranks(3.0, 1, dist, "cpu")             # one rank: no collective
        skipped = bench.run_reference(None) if rank != 0 else None     # rank 0 alone runs the oracle arm
        out[rank] = (ws, r, local, ms, single, skipped)
    finally:
        dist.destroy_process_group()


def test_step_time_is_the_slowest_rank_and_the_reference_arm_runs_on_rank_0():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    assert res[0][3] == res[1][3] == 15.0
    assert res[0][4] == res[1][4] == 3.0
    assert res[1][5] == 0
