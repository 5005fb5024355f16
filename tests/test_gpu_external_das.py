"""Core / virtual DAS subspaces with hole / particle limits (Sec. 2.4,
Fig. 1; e2_set_external_das) on the GPU against the oracle with the same
limits (pinned against the Jordan-Wigner brute force): class sizes, E2 per
root and class in both arithmetics, and the gradients dE2/dh, dE2/dc, dE2/dB
and dE2/dlambda entry by entry; the excluded determinants leave the min |D|
and the histogram."""
import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LIMITS = {
    "dcb_two_roots": (lambda: tiny_problem(6, 8, 12, 4, Lc=5, Lx=3, ham="DCB", x_scale=0.05, n_roots=2, seed=81),
                      ([2, 4], [1, 2], [4, 4, 4], [1, 2, 1])),
    "frozen_level_shift": (lambda: tiny_problem(6, 8, 14, 4, Lc=5, Lx=2, ham="DCG", x_scale=0.05, n_frozen_core=2,
                                                n_frozen_virt=2, level_shift_b=0.05, seed=82),
                           ([2, 2, 2], [1, 1, 2], [6, 8], [1, 2])),
    "das_active": (lambda: tiny_problem(4, 12, 10, 6, Lc=5, Lx=2, ham="DCB", x_scale=0.05, das_size=[4, 4, 4],
                                        das_min=[2, 0, 0], das_max=[4, 4, 2], seed=83),
                   ([4], [1], [4, 6], [1, 2])),
}


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _setup(name):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    make, lim = LIMITS[name]
    prob = make()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    o.set_external_das(*lim)
    plan = e2.E2Problem.from_problem(prob)
    plan.set_external_das(*lim)
    return e2, prob, o, c, plan, e2.device_inputs(prob, c)


@pytest.mark.parametrize("sliced", [False, True])
@pytest.mark.parametrize("name", list(LIMITS))
def test_energies_and_sizes_match_the_oracle(name, sliced):
    e2, prob, o, c, plan, t = _setup(name)
    plan.set_arithmetic(sliced)
    np.testing.assert_array_equal(plan.q_per_class, o.count_q())
    E0 = o.e0()
    e2o, eco, _ = o.e2(E0)
    E2, E2c, E0g = plan.forward(**t)
    torch.cuda.synchronize()
    np.testing.assert_allclose(E0g.cpu().numpy(), E0, rtol=0, atol=1e-10)
    np.testing.assert_allclose(E2c.cpu().numpy(), eco, rtol=0, atol=1e-9)
    np.testing.assert_allclose(E2.cpu().numpy(), e2o, rtol=0, atol=1e-9)
    code, flags, mind = plan.status()
    assert code == 0
    for cls in range(9):   # the excluded determinants never reach the smallest |D|
        if plan.q_per_class[cls] > 0:
            assert mind[0, cls] < 1e4, cls
        else:
            assert mind[0, cls] == np.inf, cls
    hist = plan.denominator_histogram(**t).cpu().numpy()
    np.testing.assert_array_equal(hist.sum(axis=1), plan.q_per_class)


@pytest.mark.parametrize("name", list(LIMITS))
def test_gradients_match_the_oracle(name):
    e2, prob, o, c, plan, t = _setup(name)
    seed = np.array([1.0, -0.6][:prob.n_roots])
    gh_o, gB_o, gw_o, gc_o = o.grad(seed=seed)
    E2, gh, gc, gbc, gbx, dl = plan.value_and_grad(seed=seed, **t)
    torch.cuda.synchronize()
    assert _rel(gh.cpu().numpy(), gh_o) < 1e-7
    assert _rel(gc.cpu().numpy(), gc_o) < 1e-7
    gB = gbc.cpu().numpy() if gbx is None else np.concatenate([gbc.cpu().numpy(), gbx.cpu().numpy()])
    assert _rel(gB, gB_o) < 1e-7
    Lc = prob.Bc.shape[0]
    dlam_o = float(np.dot(prob.wx, gw_o[Lc:])) if prob.ham != "DC" else 0.0
    assert abs(float(dl.cpu()[0]) - dlam_o) <= 1e-7 * max(abs(dlam_o), 1e-12) + 1e-15


def test_removing_the_limits_restores_the_full_space():
    e2, prob, o, c, plan, t = _setup("dcb_two_roots")
    limited = plan.forward(**t)[1].clone()
    plan.set_external_das()
    full = plan.forward(**t)[1].clone()
    ref = e2.E2Problem.from_problem(prob).forward(**t)[1]
    assert torch.equal(full, ref)
    assert not torch.equal(full, limited)
    with pytest.raises(e2.E2Error):
        plan.set_external_das([prob.n_core], [0], [], [])       # a limit of 0 is a frozen block
    with pytest.raises(e2.E2Error):
        plan.set_external_das([prob.n_core - 2], [1], [], [])   # sizes must cover the core
