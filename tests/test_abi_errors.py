"""Argument errors of the C ABI, host only: each entry point that takes
device memory checks its arguments first and returns the documented status
without enqueueing work (so these calls run on a machine without a GPU).
The device pointers passed where a check fails earlier are never read."""
import ctypes as C
import math

import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from paper_2608_11529_b300._lib import _Inputs, load
from e2_inputs import make_problem
from e2_inputs.synth import tiny_problem

OK, INVALID, SHAPE, UNSUPPORTED, WORKSPACE = 0, 1, 2, 3, 4
FAKE = 0x10000   # a non-null address that no check below lets the library read


@pytest.fixture(scope="module")
def lib():
    e2build.build()
    L = load()
    L.e2_forward.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p]
    L.e2_forward.restype = C.c_int
    L.e2_forward_noalloc.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]
    L.e2_forward_noalloc.restype = C.c_int
    return L


def _plan(**kw):
    base = dict(Lc=4, Lx=2, ham="DCB", x_scale=0.05, seed=81)
    base.update(kw)
    return e2.E2Problem.from_problem(tiny_problem(4, 8, 10, 4, **base))


def _inputs(h=FAKE, Bc=FAKE, Bx=FAKE, wx=FAKE, lam=1.0, c=FAKE):
    return _Inputs(h, Bc, Bx, wx, lam, c)


def _ws_bytes(plan):
    n = C.c_size_t()
    assert load().e2_workspace_size(plan._h, C.byref(n)) == OK
    return int(n.value)


def test_forward_argument_errors(lib):
    plan = _plan()
    need = _ws_bytes(plan)
    fwd = lambda inp, ws=FAKE * 256, nb=need, e2=FAKE: lib.e2_forward(plan._h, C.byref(inp), ws, nb, None, e2,
                                                                       None, None)
    assert lib.e2_forward(None, C.byref(_inputs()), FAKE * 256, need, None, FAKE, None, None) == INVALID
    assert fwd(_inputs(h=None)) == INVALID
    assert fwd(_inputs(c=None)) == INVALID
    assert fwd(_inputs(Bx=None)) == INVALID          # DCB needs the Breit factors and weights
    assert fwd(_inputs(lam=math.nan)) == INVALID
    assert fwd(_inputs(), e2=None) == INVALID        # no E2 output
    assert fwd(_inputs(), ws=None) == WORKSPACE
    assert fwd(_inputs(), nb=need - 256) == WORKSPACE
    assert fwd(_inputs(), ws=FAKE * 256 + 8) == WORKSPACE   # not 256-byte aligned


def test_noalloc_refuses_problems_beyond_its_scratch_before_device_work(lib):
    big = e2.E2Problem.from_problem(make_problem("ne_dcg"))   # 681 MiB of workspace
    assert _ws_bytes(big) > 32 << 20
    assert lib.e2_forward_noalloc(big._h, C.byref(_inputs()), None, FAKE, None, None) == WORKSPACE


def test_setters_and_probes_reject_out_of_range_arguments():
    L = load()
    plan = _plan()
    assert L.e2_set_shard(plan._h, 2, 2) != OK             # rank outside [0, n)
    assert L.e2_set_shard(plan._h, 0, 0) != OK
    assert L.e2_set_contraction(plan._h, 42, 1) != OK       # no such part of the path
    assert L.e2_set_class_tiles(plan._h, 99, 1) != OK
    assert L.e2_set_adjoint_chunks(None, 64, 1) == INVALID
    # probes: a class index out of range, a root out of range
    L.e2_probe_couplings.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_int, C.c_int,
                                     C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
    L.e2_probe_couplings.restype = C.c_int
    assert L.e2_probe_couplings(plan._h, None, None, 0, None, 0, 9, 0, 0, None, None, None) == INVALID
    assert L.e2_probe_couplings(plan._h, None, None, 0, None, 3, 2, 0, 0, None, None, None) == INVALID
