"""E2 as a differentiable PyTorch operation: e2_forward in the forward pass,
the hand-written adjoint e2_backward in the backward pass (V recomputed).

Gradient conventions are PyTorch's for real outputs.  For a complex input z
the gradient is dL/dRe z + i dL/dIm z.  The gradients of the Hermitian
inputs h and B^L are projected on Hermitian matrices: they give the exact
first-order change for every Hermitian perturbation, which is the only kind
these inputs admit.  The gradient of c is orthogonal to c, because E2 does
not depend on the norm of c.  lambda (the Gaunt / Breit multiplier) is
differentiable when given as a tensor.  w_x is not.
"""
from __future__ import annotations

import numpy as np

__all__ = ["E2Function", "e2_energy"]


def _function():
    import torch

    class E2Function(torch.autograd.Function):
        """apply(plan, h, B_c, c, B_x, w_x, lam) -> E2 [n_roots] (float64)."""

        @staticmethod
        def forward(ctx, plan, h, B_c, c, B_x, w_x, lam):
            lam_f = float(lam.detach().cpu()) if torch.is_tensor(lam) else float(lam)
            E2, _, _ = plan.forward(h, B_c, c, B_x=B_x, w_x=w_x, lam=lam_f)
            ctx.plan = plan
            ctx.lam = lam_f
            ctx.lam_like = lam if torch.is_tensor(lam) else None
            ctx.save_for_backward(h, B_c, c, B_x, w_x)
            return E2.clone()

        @staticmethod
        def backward(ctx, gE2):
            plan = ctx.plan
            h, B_c, c, B_x, w_x = ctx.saved_tensors
            need = ctx.needs_input_grad   # (plan, h, B_c, c, B_x, w_x, lam)
            want_B = bool(need[2] or (B_x is not None and need[4]))
            want_lambda = bool(need[6])
            seed = np.ascontiguousarray(gE2.detach().to(torch.float64).cpu().numpy())
            out = plan.backward(h, B_c, c, B_x=B_x, w_x=w_x, lam=ctx.lam, seed=seed, want_h=bool(need[1]),
                                want_c=bool(need[3]), want_B=want_B, want_lambda=want_lambda)
            gh, gc = out[0], out[1]
            gbc = out[2] if len(out) > 2 and need[2] else None
            gbx = out[3] if len(out) > 3 and need[4] else None
            glam = None
            if want_lambda and ctx.lam_like is not None:
                glam = out[4].reshape(()).to(device=ctx.lam_like.device, dtype=ctx.lam_like.dtype)
            return (None, gh if need[1] else None, gbc, gc.reshape(c.shape) if need[3] else None, gbx, None,
                    glam)

    return E2Function


_E2F = None


def E2Function():
    """The autograd.Function class (built on first use, so that importing the
    package does not import torch)."""
    global _E2F
    if _E2F is None:
        _E2F = _function()
    return _E2F


def e2_energy(plan, h, B_c, c, B_x=None, w_x=None, lam=1.0):
    """Differentiable E2 [n_roots] of a planned problem (see E2Problem)."""
    return E2Function().apply(plan, h, B_c, c, B_x, w_x, lam)
