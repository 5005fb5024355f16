"""E2 through torch.autograd: the autograd.Function's backward is the
hand-written adjoint, so torch.autograd.grad of sum_m w_m E2_m must equal
e2_backward with seed w, and dE2/dlambda must match central differences."""
import numpy as np
import pytest

from fp64_mode import fp64_contraction
from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autograd_function_gives_the_adjoint_gradients():
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = tiny_problem(4, 8, 12, 4, Lc=5, Lx=3, ham="DCB", x_scale=0.05, n_roots=2, seed=91)
    c, _ = Oracle(prob).ground_state(2)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    w = np.array([0.7, -1.3])
    h = t["h"].clone().requires_grad_(True)
    Bc = t["B_c"].clone().requires_grad_(True)
    Bx = t["B_x"].clone().requires_grad_(True)
    cc = t["c"].clone().requires_grad_(True)
    lam = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    E2 = e2.e2_energy(plan, h, Bc, cc, B_x=Bx, w_x=t["w_x"], lam=lam)
    assert torch.equal(E2.detach(), plan.forward(**t)[0])
    loss = (E2 * torch.tensor(w, device=E2.device)).sum()
    gh, gbc, gc, gbx, gl = torch.autograd.grad(loss, [h, Bc, cc, Bx, lam])
    rh, rc, rbc, rbx, rl = plan.backward(seed=w, want_B=True, want_lambda=True, **t)
    torch.cuda.synchronize()
    for a, b in ((gh, rh), (gbc, rbc), (gc, rc), (gbx, rbx)):
        assert torch.equal(a, b)
    assert float(gl) == float(rl.cpu()[0])

    def f(x):
        return float((plan.forward(**dict(t, lam=x))[0].cpu().numpy() * w).sum())
    eps = 1e-2
    with fp64_contraction(plan):
        d1 = (f(1 + eps) - f(1 - eps)) / (2 * eps)
        d2 = (f(1 + eps / 2) - f(1 - eps / 2)) / eps
    num = (4 * d2 - d1) / 3
    assert abs(float(gl) - num) <= 1e-7 * abs(num) + 1e-12, (float(gl), num)
