"""One pass for the value and its gradient, at a size where the backward GEMMs
split their contraction and the dense classes run in several tiles.

The energies that e2_backward returns must be bitwise equal to e2_forward's.
The gradient must match central differences of e2_forward along random unit
directions in h, c, every Coulomb and Breit factor, and lambda, to 1e-7 of
the gradient's norm (of the derivative itself for lambda).  The differences
are Richardson-extrapolated, so the step error is O(eps^4)."""
import numpy as np
import pytest

from fp64_mode import fp64_contraction
from e2_inputs import make_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _herm(rng, shape):
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return 0.5 * (x + np.conj(np.swapaxes(x, -1, -2)))


@pytest.fixture(scope="module")
def setup():
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = make_problem("dc_small", ham="DCB", Lx=30, x_scale=2e-3, n_roots=2)
    c, _ = Oracle(prob).ground_state(2)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    seed = np.array([1.0, -0.6])
    out = plan.value_and_grad(seed=seed, **t)
    torch.cuda.synchronize()
    return e2, prob, plan, t, seed, out


def test_backward_energies_are_bitwise_the_forward_energies(setup):
    _, _, plan, t, _, out = setup
    E2f = plan.forward(**t)[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(out[0], E2f), (out[0], E2f)


def _fd(plan, t, seed, key, direction, eps):
    """Richardson-extrapolated central difference of sum_m seed[m] E2_m."""
    def f(h):
        tt = dict(t)
        if key == "lam":
            tt["lam"] = t["lam"] + h
        else:
            tt[key] = t[key] + h * direction
        return float((plan.forward(**tt)[0].cpu().numpy() * seed).sum())
    with fp64_contraction(plan):
        d1 = (f(eps) - f(-eps)) / (2 * eps)
        d2 = (f(eps / 2) - f(-eps / 2)) / eps
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("key", ["h", "c", "B_c", "B_x", "lam"])
def test_gradient_matches_central_differences(setup, key):
    _, prob, plan, t, seed, out = setup
    _, gh, gc, gbc, gbx, dl = out
    rng = np.random.default_rng({"h": 1, "c": 2, "B_c": 3, "B_x": 4, "lam": 5}[key])
    if key == "lam":
        analytic = float(dl.cpu().numpy()[0])
        numeric = _fd(plan, t, seed, key, None, 1e-2)
        scale = max(abs(numeric), 1e-12)
    else:
        g = {"h": gh, "c": gc, "B_c": gbc, "B_x": gbx}[key].cpu().numpy()
        shape = tuple(t[key].shape)
        d = _herm(rng, shape) if key != "c" else rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        d /= np.linalg.norm(d)
        analytic = float(np.real(np.vdot(g, d)))
        eps = {"h": 1e-3, "c": 1e-3, "B_c": 1e-3, "B_x": 1e-2}[key]
        numeric = _fd(plan, t, seed, key, torch.from_numpy(d).to(t[key].device), eps)
        # the bar is relative to the gradient: ||g_a - g|| <= 1e-7 ||g|| implies, for the unit
        # direction d, |<g_a - g, d>| <= 1e-7 ||g||
        scale = max(abs(numeric), float(np.linalg.norm(g)))
    assert abs(analytic - numeric) <= 1e-7 * scale, (key, analytic, numeric, scale)
