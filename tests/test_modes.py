"""Host-side checks of the arithmetic modes (no GPU): which parts of the path
have the sliced bf16 / float-float form planned, that FP64 is the default
everywhere, that switching round-trips, and that unavailable or invalid
requests fail with the documented status codes.  Planning runs on the host
only."""
import ctypes as C

import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from e2_inputs.synth import make_problem

E2_ERR_INVALID_ARG, E2_ERR_UNSUPPORTED = 1, 3
SETUP, ADJOINT = -1, -2


@pytest.fixture(scope="module")
def plan():
    e2build.build()
    return e2.E2Problem.from_problem(make_problem("dc_small"))


def _raw(plan, cls, mode):
    return e2.load().e2_set_contraction(plan._h, cls, mode)


def test_sliced_forms_are_planned_where_the_bound_holds_and_fp64_is_the_default(plan):
    # DC 4 core + CAS(6e,12) + 40 virtual: real contraction lengths 2 K = 2 C(12,2) = 132 ((0,2), (2,0)),
    # 2 x 12 = 24 ((1,2), (2,1)), all within 256; (1,1) has 2 (1 + 12^2) = 290
    for cls in (2, 5, 6, 7, 8, SETUP, ADJOINT):
        assert plan.contraction(cls) == (False, True), cls
    assert plan.arithmetic() == "fp64"
    assert plan.contraction(4) == (False, False)      # (1,1): beyond the exact-accumulation bound
    for cls in (0, 1, 3):                             # gather classes: FP64 only
        assert plan.contraction(cls) == (False, False)


def test_modes_round_trip(plan):
    for cls in (2, 5, 6, 7, 8, SETUP, ADJOINT):
        plan.set_contraction(cls, True)
        assert plan.contraction(cls) == (True, True)
        plan.set_contraction(cls, False)
        assert plan.contraction(cls) == (False, True)
    plan.set_arithmetic(True)
    assert plan.arithmetic() == "sliced"
    assert all(plan.contraction(cls) == (True, True) for cls in (2, 5, 6, 7, 8, SETUP, ADJOINT))
    assert plan.contraction(4) == (False, False)
    plan.set_arithmetic(False)
    assert plan.arithmetic() == "fp64"


def test_unavailable_and_invalid_requests(plan):
    assert _raw(plan, 4, 1) == E2_ERR_UNSUPPORTED     # sliced (1,1)
    assert _raw(plan, 4, 0) == 0                      # FP64 is always available
    assert _raw(plan, 2, 2) == E2_ERR_INVALID_ARG     # no such mode
    assert _raw(plan, 9, 0) == E2_ERR_INVALID_ARG     # no such class
    assert _raw(plan, -3, 0) == E2_ERR_INVALID_ARG
    mode, avail = C.c_int(7), C.c_int(7)
    assert e2.load().e2_contraction(None, 2, C.byref(mode), C.byref(avail)) == E2_ERR_INVALID_ARG
    assert e2.load().e2_contraction(plan._h, 2, None, None) == 0   # both outputs optional


def test_adjoint_chunk_setter(plan):
    lib = e2.load()
    assert lib.e2_set_adjoint_chunks(plan._h, 64, 1) == 0
    assert lib.e2_set_adjoint_chunks(plan._h, 0, 0) == 0             # back to the plan's values
    assert lib.e2_set_adjoint_chunks(None, 64, 1) == E2_ERR_INVALID_ARG


def test_sliced_buffers_are_gated_by_size():
    # the Xe shape's slices and float-float tables exceed 16 GiB: no sliced classes; the setup and adjoint
    # products keep their (opt-in) sliced form
    p = e2.E2Problem(46, 24, 1000, 8, ham="DCB", L_coulomb=1400, L_extra=700)
    for cls in (2, 5, 6, 7, 8):
        assert p.contraction(cls) == (False, False), cls
    assert p.contraction(SETUP) == (False, True)
    assert p.contraction(ADJOINT) == (False, True)
