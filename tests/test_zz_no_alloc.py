"""e2_forward_noalloc: the allocation-free variant for callers that cannot
call cudaMalloc (graph capture, host programs owning the allocator).  It must
give the same energies as e2_forward with a caller workspace, call after call,
although every call reuses the one scratch array inside the library.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest

from e2_inputs import make_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E2_ERR_WORKSPACE = 4


def _lib():
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import _lib as binding
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    lib = C.CDLL(e2.LIB_PATH)
    lib.e2_forward_noalloc.argtypes = [C.c_void_p, C.POINTER(binding._Inputs), C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p]
    lib.e2_forward_noalloc.restype = C.c_int
    return e2, binding, lib


def _inputs(binding, plan, t):
    return binding._Inputs(t["h"].data_ptr(), t["B_c"].data_ptr(),
                           t["B_x"].data_ptr() if plan.L_extra else None,
                           t["w_x"].data_ptr() if plan.L_extra else None, float(t["lam"]), t["c"].data_ptr())


def test_noalloc_forward_matches_workspace_forward_on_consecutive_calls():
    from oracle import Oracle
    e2, binding, lib = _lib()
    prob = make_problem("dc_small")
    c, _ = Oracle(prob).ground_state(1)
    plan = e2.E2Problem.from_problem(prob)
    t = e2.device_inputs(prob, c)
    ref = [x.clone() for x in plan.forward(**t)]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = (torch.full((1,), np.nan, dtype=torch.float64, device="cuda"),
               torch.full((1, 9), np.nan, dtype=torch.float64, device="cuda"),
               torch.full((1,), np.nan, dtype=torch.float64, device="cuda"))
        inp = _inputs(binding, plan, t)
        st = lib.e2_forward_noalloc(plan._h, C.byref(inp), C.c_void_p(stream), out[0].data_ptr(),
                                    out[1].data_ptr(), out[2].data_ptr())
        assert st == 0, e2.load().e2_status_string(st)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out[1].cpu().numpy(), ref[1].cpu().numpy(), rtol=0, atol=1e-9)
        np.testing.assert_allclose(out[0].cpu().numpy(), ref[0].cpu().numpy(), rtol=0, atol=1e-9)
        np.testing.assert_allclose(out[2].cpu().numpy(), ref[2].cpu().numpy(), rtol=0, atol=1e-10)


def test_noalloc_rejects_problems_larger_than_the_static_scratch():
    e2, binding, lib = _lib()
    plan = e2.E2Problem(2, 16, 200, 8, ham="DCG", L_coulomb=400, L_extra=200)   # ~275 MB of scratch
    assert plan.workspace_bytes > (32 << 20)
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    inp = binding._Inputs(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 1.0,
                          dummy.data_ptr())
    st = lib.e2_forward_noalloc(plan._h, C.byref(inp), None, dummy.data_ptr(), None, None)
    assert st == E2_ERR_WORKSPACE
