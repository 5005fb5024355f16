"""Batched evaluation: one persistent launch for every class of several jobs
(different Hamiltonians, root counts, frozen cutoffs, a CAS and a DAS
reference), plain and captured in a CUDA graph, against e2_forward job by job
(bitwise: same partial slots, same reduction order) and the oracle."""
import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _jobs():
    base = dict(n_core=6, n_act=10, n_virt=16, n_elec=5, Lc=6, Lx=3, x_scale=0.05, seed=61)
    specs = [dict(ham="DC", n_roots=1), dict(ham="DCG", n_roots=2, n_frozen_core=2),
             dict(ham="DCB", n_roots=2, n_frozen_core=2, n_frozen_virt=4),
             dict(ham="DCB", n_roots=1, das_size=[4, 6], das_min=[2, 0], das_max=[4, 3], n_frozen_virt=2)]
    out = []
    for sp in specs:
        kw = dict(base)
        kw.update(sp)
        p = tiny_problem(**kw)
        o = Oracle(p)
        c, _ = o.ground_state(p.n_roots)
        out.append((p, o, c))
    return out


@pytest.mark.parametrize("roots_per_launch", [0, 1])
@pytest.mark.parametrize("col_tiles", [False, True])
@pytest.mark.parametrize("sliced", [True, False])
def test_batch_matches_single_forward_and_oracle_and_replays_in_a_graph(col_tiles, sliced, roots_per_launch):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    jobs = _jobs()
    plans = [e2.E2Problem.from_problem(p) for p, _, _ in jobs]
    for plan in plans:                             # plain columns, or compacted tiles where a plan exists
        for cls in (2, 4, 5, 6):
            if plan.class_tiles(cls)[0]:
                plan.set_class_tiles(cls, col_tiles)
        for cls in (-1, 2, 5, 6, 7, 8):            # sliced classes run beside the persistent FP64 kernel
            if plan.contraction(cls)[1]:
                plan.set_contraction(cls, sliced)
    inputs = [e2.device_inputs(p, c) for p, _, c in jobs]
    single = []
    for plan, t in zip(plans, inputs):
        E2, E2c, _ = plan.forward(**t)
        single.append((E2.clone(), E2c.clone()))
    # roots_per_launch = 1: the two-root jobs run in two persistent launches
    # that reuse one coupling-table slot per job
    batch = e2.E2Batch(plans, roots_per_launch=roots_per_launch)
    batch.prepare(torch.device("cuda"))
    out = batch.forward(inputs)
    torch.cuda.synchronize()
    for (E2, E2c), (B2, B2c), (p, o, c) in zip(single, out, jobs):
        assert torch.equal(E2, B2) and torch.equal(E2c, B2c)
        _, ec, _ = o.e2()
        np.testing.assert_allclose(B2c.cpu().numpy(), ec, rtol=0, atol=1e-9)
    # capture once, replay twice
    for o2 in out:
        o2[0].zero_()
        o2[1].zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            batch.forward(inputs)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for o2 in out:
            o2[0].zero_()
        g.replay()
        torch.cuda.synchronize()
        for (E2, E2c), (B2, B2c) in zip(single, out):
            assert torch.equal(E2, B2) and torch.equal(E2c, B2c)
    assert batch.launch_count() > 0


@pytest.mark.parametrize("sliced", [False, True])
def test_batch_backward_equals_each_jobs_backward(sliced):
    """e2_batch_backward: every job's energies and gradients bitwise equal to
    its own e2_backward, and the energies to its forward."""
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    jobs = _jobs()
    plans = [e2.E2Problem.from_problem(p) for p, _, _ in jobs]
    for plan in plans:
        plan.set_arithmetic(sliced)
    inputs = [e2.device_inputs(p, c) for p, _, c in jobs]
    seeds = [np.linspace(1.0, 0.5, p.n_roots) for p, _, _ in jobs]
    ref = []
    for plan, t, sd in zip(plans, inputs, seeds):
        E2f = plan.forward(**t)[0].clone()
        out = plan.value_and_grad(**t, seed=sd)
        ref.append((E2f, [x.clone() if x is not None else None for x in out]))
    batch = e2.E2Batch(plans)
    got = batch.backward(inputs, seeds=seeds)
    torch.cuda.synchronize()
    for (E2f, r), g in zip(ref, got):
        assert torch.equal(g[0], E2f) and torch.equal(g[0], r[0])
        for k in range(1, 6):
            if r[k] is not None and g[k] is not None:
                assert torch.equal(g[k], r[k]), k
