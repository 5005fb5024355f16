"""Batch workspace layout, host only: with root groups
(e2_batch_set_roots_per_launch) each job keeps one coupling-table slot per
root of a launch instead of one per root, so the workspace shrinks by the
table slots it no longer holds and never grows; a negative group size is
refused; jobs with fewer roots than the group size keep all of theirs; and
E2Batch.plan_batches splits jobs into batches that fit a memory budget."""
import ctypes as C

import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from paper_2608_11529_b300._lib import load
from e2_inputs.synth import tiny_problem


def _plans():
    e2build.build()
    specs = [dict(ham="DC", n_roots=3), dict(ham="DCB", Lx=3, x_scale=0.05, n_roots=2, n_frozen_core=2),
             dict(ham="DCG", Lx=2, x_scale=0.05, n_roots=1)]
    return [e2.E2Problem.from_problem(tiny_problem(6, 10, 16, 5, Lc=6, seed=71 + i, **sp))
            for i, sp in enumerate(specs)]


def _ws(plans, k):
    return e2.E2Batch(plans, roots_per_launch=k).workspace_bytes


def test_root_groups_shrink_the_batch_workspace():
    plans = _plans()
    full = _ws(plans, 0)
    one = _ws(plans, 1)
    two = _ws(plans, 2)
    assert one < two < full
    # k at least the largest root count: every root in one launch, the same layout
    assert _ws(plans, 3) == full and _ws(plans, 8) == full


def test_negative_root_group_is_refused():
    plans = _plans()
    b = e2.E2Batch(plans)
    st = load().e2_batch_set_roots_per_launch(b._h, C.c_int(-1))
    assert st != 0
    with pytest.raises(e2.E2Error):
        e2.E2Batch(plans, roots_per_launch=-2)


def test_plan_batches_fits_the_budget():
    plans = _plans()
    one = [_ws([p], 1) for p in plans]
    # a budget that holds the first two jobs with one slot each, not all three
    budget = _ws(plans[:2], 1) + 1
    assert _ws(plans, 1) > budget
    out = e2.E2Batch.plan_batches(plans, budget)
    assert [len(g) for g, _ in out] == [2, 1]
    assert sum(len(g) for g, _ in out) == len(plans)
    for g, k in out:
        assert _ws(g, k) <= budget
        if k:   # the largest group size that fits
            assert k == max(p.n_roots for p in g) or _ws(g, k + 1) > budget
    # a budget for everything at once: one batch, every root in one launch
    out = e2.E2Batch.plan_batches(plans, _ws(plans, 0))
    assert len(out) == 1 and out[0][1] == 0
    # a job that cannot fit alone
    with pytest.raises(e2.E2Error):
        e2.E2Batch.plan_batches(plans, min(one) - 1)
