"""Sharding of the external space over ranks, host side (no GPU): every
class's units split into contiguous, disjoint, balanced shares that cover
them exactly once, for 1 to 8 ranks; and, with two gloo ranks on the CPU,
that the per-tile partial slots the ranks own (from the documented slot
layout) cover the whole partial set exactly once, so the element-wise sum of
the ranks' partials is the unsharded set."""
import os
import socket
import sys

import numpy as np
import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from e2_inputs import make_problem
from e2_inputs.synth import tiny_problem

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PLANS = {
    "dc_small": lambda: make_problem("dc_small"),
    "das_three": lambda: tiny_problem(4, 12, 10, 6, Lc=5, Lx=2, ham="DCB", das_size=[4, 4, 4], das_min=[2, 0, 0],
                                      das_max=[4, 4, 2], n_roots=2, seed=23),
    "ne_dcg": lambda: make_problem("ne_dcg", Lc=2, Lx=1),
    "ar_dcb_das": lambda: make_problem("ar_dcb_das", Lc=2, Lx=1),
}


def _plan(name):
    e2build.build()
    return e2.E2Problem.from_problem(PLANS[name]())


@pytest.mark.parametrize("name", list(PLANS))
def test_shares_cover_every_unit_once(name):
    plan = _plan(name)
    for n in range(1, 9):
        for cls in range(9):
            got = []
            for r in range(n):
                plan.set_shard(r, n)
                units, a, b = plan.shard_units(cls)
                assert 0 <= a <= b <= units
                got.append((a, b))
            assert got[0][0] == 0 and got[-1][1] == units
            assert all(got[k][1] == got[k + 1][0] for k in range(n - 1))         # contiguous, disjoint
            sizes = [b - a for a, b in got]
            assert max(sizes) - min(sizes) <= 1                                    # balanced
    plan.set_shard(0, 1)
    assert all(plan.shard_units(cls)[1:] == (0, plan.shard_units(cls)[0]) for cls in range(9))


def test_invalid_shards_are_rejected():
    plan = _plan("dc_small")
    lib = e2.load()
    assert lib.e2_set_shard(plan._h, 2, 2) == 1
    assert lib.e2_set_shard(plan._h, -1, 2) == 1
    assert lib.e2_set_shard(plan._h, 0, 0) == 1
    assert lib.e2_set_shard(None, 0, 1) == 1


def _owned_slots(plan, prob):
    """Partial slots (all roots, classes; the documented layout) of this rank."""
    from math import comb
    nc = sum(1 for k in range(prob.n_core) if not prob.frozen[k])
    nv = sum(1 for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v])
    nvb = (nv + 7) // 8
    slots = []
    off = 0
    counts = []
    for cls in range(9):
        units, a, b = plan.shard_units(cls)
        q = plan.q_per_class[cls]
        if units == 0:
            counts.append(([], 0))
            continue
        if cls in (2, 4, 5, 6, 7):              # dense: partial[tile_n * rt + tile_m], tiles of 64 x 64
            rows = {2: comb(nv, 2), 4: nc * nv, 5: nc * comb(nv, 2), 6: comb(nc, 2), 7: comb(nc, 2) * nv}[cls]
            nA = int(round(q / rows))
            rt, ct = units, (nA + 63) // 64
            mine = [tn * rt + tm for tn in range(ct) for tm in range(a, b)]
            counts.append((mine, rt * ct))
        elif cls == 8:                          # (2,2): partial[u * A blocks + x], u = z nyb + y
            nA = int(round(q / (comb(nc, 2) * comb(nv, 2))))
            gx = (nA + 255) // 256
            mine = [u * gx + x for u in range(a, b) for x in range(gx)]
            counts.append((mine, units * gx))
        elif cls in (1, 3):                     # rows x 256-string blocks
            rows = nv if cls == 1 else nc
            nA = int(round(q / rows))
            gx = (nA + 255) // 256
            mine = [r * gx + x for r in range(a, b) for x in range(gx)]
            counts.append((mine, rows * gx))
        else:                                   # (0,0): string blocks
            mine = list(range(a, b))
            counts.append((mine, units))
    total_per_root = sum(cnt for _, cnt in counts)
    for r in range(plan.n_roots):
        base = r * total_per_root
        o = 0
        for mine, cnt in counts:
            slots += [base + o + s for s in mine]
            o += cnt
    return np.array(slots, np.int64), total_per_root * plan.n_roots


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, name, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        plan = _plan(name)
        plan.set_shard(rank, world)
        slots, total = _owned_slots(plan, PLANS[name]())
        part = torch.zeros(total, dtype=torch.float64)
        part[torch.from_numpy(slots)] = torch.from_numpy(slots.astype(np.float64) + 1.0)
        count = torch.zeros(total, dtype=torch.float64)
        count[torch.from_numpy(slots)] = 1.0
        dist.all_reduce(part)
        dist.all_reduce(count)
        out[rank] = (bool(torch.equal(part, torch.arange(1, total + 1, dtype=torch.float64))),
                     bool(torch.all(count == 1.0)), total)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", ["das_three", "ne_dcg"])
def test_two_ranks_cover_every_partial_slot_once(name):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, name, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] and res[0][1] and res[1][0] and res[1][1]
    assert res[0][2] == res[1][2] > 0
