"""Sharded forward on one GPU: the ranks' shares run one after another (each
e2_forward with e2_set_shard writes only its own partial slots), their
partials are summed element-wise and their smallest-|D| keys minimised, as the
ranks' collective would, and e2_reduce then gives E2, E2_class and the status
bitwise equal to the unsharded forward, for 1 to 5 ranks.  (Ranks that wait on
one another are never emulated on one GPU; nothing here waits.)"""
import numpy as np
import pytest

from e2_inputs import make_problem
from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "dc_small": lambda: make_problem("dc_small"),
    "das_three_two_roots": lambda: tiny_problem(4, 12, 10, 6, Lc=5, Lx=2, ham="DCB", x_scale=0.05,
                                                das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2],
                                                n_roots=2, seed=23),
    "level_shift_frozen": lambda: tiny_problem(6, 8, 14, 4, Lc=6, Lx=4, ham="DCG", x_scale=0.05,
                                               n_frozen_core=2, n_frozen_virt=3, level_shift_b=0.05, seed=31),
}


@pytest.mark.parametrize("sliced", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_sharded_partials_sum_to_the_unsharded_forward(name, sliced):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = CASES[name]()
    c, _ = Oracle(prob).ground_state(prob.n_roots)
    plan = e2.E2Problem.from_problem(prob)
    plan.set_arithmetic(sliced)
    t = e2.device_inputs(prob, c)
    E2, E2c, E0 = [x.clone() for x in plan.forward(**t)]
    ref_status = plan.status()
    for n in (1, 2, 3, 5):
        acc, keys = None, None
        for r in range(n):
            plan.set_shard(r, n)
            plan.forward(**t)
            part, k = plan.shard_buffers()
            acc = part.clone() if acc is None else acc + part
            keys = k.clone() if keys is None else torch.minimum(keys, k)
        part, k = plan.shard_buffers()
        part.copy_(acc)
        k.copy_(keys)
        got = plan.reduce()
        torch.cuda.synchronize()
        assert torch.equal(got[0], E2) and torch.equal(got[1], E2c) and torch.equal(got[2], E0), n
        st = plan.status()
        assert st[:2] == ref_status[:2] and np.array_equal(st[2], ref_status[2]), n
    plan.set_shard(0, 1)


def test_backward_refuses_a_sharded_problem():
    import paper_2608_11529_b300 as e2
    prob = make_problem("dc_small")
    c, _ = Oracle(prob).ground_state(1)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    plan.set_shard(1, 2)
    with pytest.raises(e2.E2Error):
        plan.value_and_grad(**t)
    plan.set_shard(0, 1)
    plan.value_and_grad(**t)


def test_checkpointed_run_resumes_bitwise(tmp_path):
    """A run in 4 resumable parts, stopped after 2 and resumed by a fresh plan
    (as a new process would), gives E2 bitwise equal to the one-piece
    forward; a directory of another run is refused."""
    import paper_2608_11529_b300 as e2
    prob = CASES["das_three_two_roots"]()
    c, _ = Oracle(prob).ground_state(prob.n_roots)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    ref = [x.clone() for x in plan.forward(**t)]
    path = str(tmp_path / "ckpt")
    assert plan.checkpointed_forward(path, **t, pieces=4, max_pieces=2, tag="das3") is None
    fresh = e2.E2Problem.from_problem(prob)
    got = fresh.checkpointed_forward(path, **t, pieces=4, tag="das3")
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    again = e2.E2Problem.from_problem(prob).checkpointed_forward(path, **t, pieces=4, tag="das3")  # all saved
    assert all(torch.equal(a, b) for a, b in zip(again, ref))
    with pytest.raises(e2.E2Error):
        fresh.checkpointed_forward(path, **t, pieces=3, tag="das3")
