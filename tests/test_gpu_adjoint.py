"""GPU adjoint against the oracle's gradient: dE2/dh (Hermitian-projected,
the unrelaxed response one-particle density) and dE2/dc per root, entry by
entry, on the same seeded inputs; relative error <= 1e-7 of the largest
entry (the gradient bar), and <c|cbar> = 0."""
import numpy as np
import pytest

from fp64_mode import fp64_contraction
from e2_inputs import make_problem
from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    "dcb_roots_frozen": lambda: tiny_problem(4, 8, 10, 4, Lc=5, Lx=3, ham="DCB", x_scale=0.05, n_roots=2,
                                             n_frozen_core=2, n_frozen_virt=2, seed=51),
    "dcg_odd": lambda: tiny_problem(4, 8, 8, 3, Lc=4, Lx=2, ham="DCG", x_scale=0.05, seed=52),
    "das": lambda: tiny_problem(2, 8, 8, 4, Lc=4, das_size=[4, 4], das_min=[1, 1], das_max=[3, 3], seed=53),
    "level_shift": lambda: tiny_problem(4, 6, 10, 3, Lc=4, level_shift_b=0.05, seed=54),
    "mid_dcb": lambda: tiny_problem(4, 10, 18, 5, Lc=6, Lx=3, ham="DCB", x_scale=0.05, seed=55),
    # 24 active spinors, as in the Ar- to Xe-shaped workloads (the per-row
    # occupation sums then run at another block size)
    "wide_active": lambda: tiny_problem(4, 24, 6, 3, Lc=4, Lx=2, ham="DCB", x_scale=0.05, seed=56),
}


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_matches_oracle_gradient(name):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = CASES[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    c = c * (1.0 + 0.5j)                              # unnormalised reference
    o.set_c(c)
    seed = np.array([1.0, -0.6][:prob.n_roots])
    gh_o, _, _, gc_o = o.grad(seed=seed)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    gh, gc = plan.backward(seed=seed, **t)
    torch.cuda.synchronize()
    gh, gc = gh.cpu().numpy(), gc.cpu().numpy()
    assert _rel(gh, gh_o) < 1e-7, _rel(gh, gh_o)
    assert _rel(gc, gc_o) < 1e-7, _rel(gc, gc_o)
    for m in range(prob.n_roots):
        assert abs(np.vdot(c[m], gc[m])) < 1e-9 * np.abs(gc[m]).max() * np.abs(c[m]).max() * c.shape[1]


@pytest.mark.parametrize("name", list(CASES))
def test_factor_gradient_and_breit_derivative_match_oracle(name):
    """dE2/dB^L for every Coulomb and Gaunt/Breit factor (Hermitian-projected)
    and dE2/dlambda against the oracle's explicit accumulation."""
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = CASES[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    o.set_c(c)
    seed = np.array([1.0, -0.6][:prob.n_roots])
    _, gB_o, gw_o, _ = o.grad(seed=seed)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    gh, gc, gbc, gbx, dl = plan.backward(seed=seed, want_B=True, want_lambda=True, **t)
    torch.cuda.synchronize()
    Lc = prob.Bc.shape[0]
    gB = gbc.cpu().numpy() if gbx is None else np.concatenate([gbc.cpu().numpy(), gbx.cpu().numpy()])
    assert _rel(gB, gB_o) < 1e-7, _rel(gB, gB_o)
    dlam_o = float(np.dot(prob.wx, gw_o[Lc:])) if prob.ham != "DC" else 0.0
    assert abs(float(dl.cpu()[0]) - dlam_o) <= 1e-7 * max(abs(dlam_o), 1e-12) + 1e-15


@pytest.mark.parametrize("name", ["mid_dcb", "das"])
def test_adjoint_with_column_tiles_matches_oracle(name):
    """The adjoint class kernel over compacted column tiles (amplitudes and
    denominator weights scattered back to their strings) gives the oracle's
    dE2/dh, dE2/dc and dE2/dB."""
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = CASES[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    o.set_c(c)
    seed = np.array([1.0, -0.6][:prob.n_roots])
    gh_o, gB_o, _, gc_o = o.grad(seed=seed)
    plan = e2.E2Problem.from_problem(prob)
    on = [cls for cls in (2, 4, 5, 6) if plan.class_tiles(cls)[0]]
    assert on
    for cls in on:
        plan.set_class_tiles(cls, True)
    t = e2.device_inputs(prob, c)
    E2, gh, gc, gbc, gbx, _ = plan.value_and_grad(seed=seed, **t)
    torch.cuda.synchronize()
    assert torch.equal(E2, plan.forward(**t)[0])
    gB = gbc.cpu().numpy() if gbx is None else np.concatenate([gbc.cpu().numpy(), gbx.cpu().numpy()])
    assert _rel(gh.cpu().numpy(), gh_o) < 1e-7
    assert _rel(gc.cpu().numpy(), gc_o) < 1e-7
    assert _rel(gB, gB_o) < 1e-7


@pytest.mark.parametrize("name", ["mid_dcb", "dcb_roots_frozen"])
def test_adjoint_in_smallest_chunks(name):
    """The adjoint in 64-row chunks of every dense class and one core pair per
    class-(2,2) chunk: per-tile sums reduced chunk by chunk give the oracle's
    gradients (default, sliced products), and, with every product in FP64,
    the planned single-chunk gradients up to summation order; the forward's
    E2 bit for bit.  (Sliced products cut each chunk with its own scales, so
    between chunkings they agree to the slices' precision, not to rounding.)"""
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = CASES[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    o.set_c(c)
    seed = np.array([1.0, -0.6][:prob.n_roots])
    gh_o, gB_o, _, gc_o = o.grad(seed=seed)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    plan.set_adjoint_chunks(rows=64, core_pairs=1)
    E2, gh, gc, gbc, gbx, dl = plan.value_and_grad(seed=seed, **t)
    torch.cuda.synchronize()
    assert torch.equal(E2, plan.forward(**t)[0])
    gB = gbc.cpu().numpy() if gbx is None else np.concatenate([gbc.cpu().numpy(), gbx.cpu().numpy()])
    assert _rel(gh.cpu().numpy(), gh_o) < 1e-7
    assert _rel(gc.cpu().numpy(), gc_o) < 1e-7
    assert _rel(gB, gB_o) < 1e-7
    with fp64_contraction(plan):
        plan.set_adjoint_chunks()
        ref = plan.value_and_grad(seed=seed, **t)
        plan.set_adjoint_chunks(rows=64, core_pairs=1)
        out = plan.value_and_grad(seed=seed, **t)
        plan.set_adjoint_chunks()
    torch.cuda.synchronize()
    for k in (1, 2, 3, 5):  # g_h, g_c, g_Bc, dE2/dlambda
        a, b = out[k], ref[k]
        assert _rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12, k
