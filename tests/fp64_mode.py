"""Finite differences of E2 need a function smooth to well below the size of
the differenced change.  The sliced bf16 contraction rounds each V near 2^-40
of its row and string scale (E2 to about 1e-13 relative), which a central
difference over a 1e-9 change turns into a visible error; the FP64
contraction is smooth to rounding.  The adjoint forms its amplitudes in FP64
either way, so the finite differences that check it use this mode."""
from contextlib import contextmanager

DENSE_SLICED = (-2, -1, 2, 5, 6, 7, 8)  # -1, -2: the setup and adjoint products; 8: class (2,2)


@contextmanager
def fp64_contraction(plan):
    saved = {cls: plan.contraction(cls)[0] for cls in DENSE_SLICED}
    for cls in DENSE_SLICED:
        plan.set_contraction(cls, False)
    try:
        yield plan
    finally:
        for cls, on in saved.items():
            if on:
                plan.set_contraction(cls, True)
