"""ctypes binding of libe2.so (argument marshalling only).

Every computation runs in the library's sm_103a kernels; this module builds
the descriptor, allocates caller-owned device memory with PyTorch and passes
raw pointers.  It raises if the library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libe2.so")
NCLASS = 9
HAM = {"DC": 0, "DCG": 1, "DCB": 2}
CLASS_NAMES = ["(0,0)", "(0,1)", "(0,2)", "(1,0)", "(1,1)", "(1,2)", "(2,0)", "(2,1)", "(2,2)"]


class _Desc(C.Structure):
    _fields_ = [("n_core", C.c_int32), ("n_active", C.c_int32), ("n_virt", C.c_int32), ("n_elec", C.c_int32),
                ("frozen", C.POINTER(C.c_uint8)), ("n_das", C.c_int32), ("das_size", C.POINTER(C.c_int32)),
                ("das_min", C.POINTER(C.c_int32)), ("das_max", C.POINTER(C.c_int32)), ("ham", C.c_int32),
                ("L_coulomb", C.c_int32), ("L_extra", C.c_int32), ("n_roots", C.c_int32),
                ("level_shift_b", C.c_double), ("class_mask", C.c_uint32)]


class _Inputs(C.Structure):
    _fields_ = [("h", C.c_void_p), ("B_c", C.c_void_p), ("B_x", C.c_void_p), ("w_x", C.c_void_p),
                ("lam", C.c_double), ("c", C.c_void_p)]


_lib = None


def load():
    """Load libe2.so (raises OSError when it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libe2.so not built: run `python -m paper_2608_11529_b300.build` ({LIB_PATH})")
        L = C.CDLL(LIB_PATH)
        L.e2_problem_create.argtypes = [C.POINTER(_Desc), C.POINTER(C.c_void_p)]
        L.e2_problem_create.restype = C.c_int
        L.e2_problem_destroy.argtypes = [C.c_void_p]
        L.e2_problem_destroy.restype = C.c_int
        L.e2_problem_info.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]
        L.e2_problem_info.restype = C.c_int
        L.e2_workspace_size.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
        L.e2_workspace_size.restype = C.c_int
        L.e2_forward.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
        L.e2_forward.restype = C.c_int
        L.e2_reference_workspace_size.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
        L.e2_reference_workspace_size.restype = C.c_int
        L.e2_reference_solve.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_double, C.c_int, C.c_void_p, C.c_size_t,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
        L.e2_reference_solve.restype = C.c_int
        L.e2_partials.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_void_p),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_void_p)]
        L.e2_partials.restype = C.c_int
        L.e2_class_tiles.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int)]
        L.e2_class_tiles.restype = C.c_int
        L.e2_class_tiles_copy.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.e2_class_tiles_copy.restype = C.c_int
        L.e2_set_class_tiles.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.e2_set_class_tiles.restype = C.c_int
        L.e2_set_adjoint_chunks.argtypes = [C.c_void_p, C.c_int64, C.c_int]
        L.e2_set_adjoint_chunks.restype = C.c_int
        L.e2_set_contraction.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.e2_set_contraction.restype = C.c_int
        L.e2_contraction.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.e2_contraction.restype = C.c_int
        L.e2_autotune.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
        L.e2_autotune.restype = C.c_int
        L.e2_backward_workspace_size.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
        L.e2_backward_workspace_size.restype = C.c_int
        L.e2_backward.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.e2_backward.restype = C.c_int
        L.e2_batch_create.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
        L.e2_batch_create.restype = C.c_int
        L.e2_batch_destroy.argtypes = [C.c_void_p]
        L.e2_batch_destroy.restype = C.c_int
        L.e2_batch_workspace_size.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
        L.e2_batch_workspace_size.restype = C.c_int
        L.e2_batch_prepare.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
        L.e2_batch_prepare.restype = C.c_int
        L.e2_batch_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p,
                                       C.c_void_p]
        L.e2_batch_forward.restype = C.c_int
        L.e2_batch_launch_count.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
        L.e2_batch_launch_count.restype = C.c_int
        L.e2_batch_set_roots_per_launch.argtypes = [C.c_void_p, C.c_int]
        L.e2_batch_set_roots_per_launch.restype = C.c_int
        L.e2_launch_count.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
        L.e2_launch_count.restype = C.c_int
        L.e2_profile_events.argtypes = [C.c_void_p, C.c_void_p]
        L.e2_profile_events.restype = C.c_int
        L.e2_fp64_peak.argtypes = [C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.e2_fp64_peak.restype = C.c_int
        L.e2_query_status.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_uint32), C.c_void_p]
        L.e2_query_status.restype = C.c_int
        L.e2_coupling_tables.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p,
                                         C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]
        L.e2_coupling_tables.restype = C.c_int
        L.e2_probe_couplings.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p,
                                         C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
        L.e2_probe_couplings.restype = C.c_int
        L.e2_set_shard.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.e2_set_shard.restype = C.c_int
        L.e2_shard_units.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]
        L.e2_shard_units.restype = C.c_int
        L.e2_shard_buffers.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]
        L.e2_shard_buffers.restype = C.c_int
        L.e2_reduce.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.e2_reduce.restype = C.c_int
        L.e2_form_integrals.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p]
        L.e2_form_integrals.restype = C.c_int
        L.e2_tuning_save.argtypes = [C.c_void_p, C.c_char_p]
        L.e2_tuning_save.restype = C.c_int
        L.e2_tuning_load.argtypes = [C.c_void_p, C.c_char_p]
        L.e2_tuning_load.restype = C.c_int
        L.e2_batch_backward_workspace_size.argtypes = [C.c_void_p, C.POINTER(C.c_size_t)]
        L.e2_batch_backward_workspace_size.restype = C.c_int
        L.e2_batch_backward.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p] + \
            [C.c_void_p] * 6
        L.e2_batch_backward.restype = C.c_int
        L.e2_denominator_histogram.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p,
                                               C.c_int, C.c_void_p]
        L.e2_denominator_histogram.restype = C.c_int
        L.e2_prepare_roots.argtypes = [C.c_void_p, C.POINTER(_Inputs), C.c_void_p, C.c_size_t, C.c_void_p]
        L.e2_prepare_roots.restype = C.c_int
        L.e2_set_external_das.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                          C.c_void_p]
        L.e2_set_external_das.restype = C.c_int
        L.e2_status_string.argtypes = [C.c_int]
        L.e2_status_string.restype = C.c_char_p
        _lib = L
    return _lib


class E2Error(RuntimeError):
    pass


def _check(st):
    if st != 0:
        raise E2Error(load().e2_status_string(st).decode())


class E2Problem:
    """A planned E2 evaluation (host plan of ``e2_problem_create``)."""

    def __init__(self, n_core, n_active, n_virt, n_elec, *, frozen=None, das_size=None, das_min=None, das_max=None,
                 ham="DC", L_coulomb=1, L_extra=0, n_roots=1, level_shift_b=0.0, class_mask=0x1FF):
        L = load()
        n = n_core + n_active + n_virt
        if das_size is None:
            das_size, das_min, das_max = [n_active], [n_elec], [n_elec]
        self._frozen = np.ascontiguousarray(np.zeros(n, np.uint8) if frozen is None else frozen, np.uint8)
        self._ds = np.ascontiguousarray(das_size, np.int32)
        self._dmin = np.ascontiguousarray(das_min, np.int32)
        self._dmax = np.ascontiguousarray(das_max, np.int32)
        d = _Desc(n_core, n_active, n_virt, n_elec, self._frozen.ctypes.data_as(C.POINTER(C.c_uint8)), len(das_size),
                  self._ds.ctypes.data_as(C.POINTER(C.c_int32)), self._dmin.ctypes.data_as(C.POINTER(C.c_int32)),
                  self._dmax.ctypes.data_as(C.POINTER(C.c_int32)), HAM[ham] if isinstance(ham, str) else int(ham),
                  L_coulomb, L_extra, n_roots, float(level_shift_b), int(class_mask))
        h = C.c_void_p()
        _check(L.e2_problem_create(C.byref(d), C.byref(h)))
        self._h = h
        self.n = n
        self.n_roots = n_roots
        self.L_extra = L_extra
        n_p = C.c_int64()
        q = np.zeros(NCLASS)
        _check(L.e2_problem_info(self._h, C.byref(n_p), q.ctypes.data_as(C.c_void_p)))
        self.n_p = int(n_p.value)
        self.q_per_class = q
        ws = C.c_size_t()
        _check(L.e2_workspace_size(self._h, C.byref(ws)))
        self.workspace_bytes = int(ws.value)
        _check(L.e2_reference_workspace_size(self._h, C.byref(ws)))
        self.solve_workspace_bytes = int(ws.value)
        _check(L.e2_backward_workspace_size(self._h, C.byref(ws)))
        self.backward_workspace_bytes = int(ws.value)
        self._ws = None
        self._events = None

    @classmethod
    def from_problem(cls, prob, class_mask=0x1FF, n_roots=None, level_shift_b=None):
        """Plan for an ``e2_inputs.Problem``."""
        Lx = prob.Bx.shape[0] if prob.ham != "DC" else 0
        return cls(prob.n_core, prob.n_act, prob.n_virt, prob.n_elec, frozen=prob.frozen, das_size=prob.das_size,
                   das_min=prob.das_min, das_max=prob.das_max, ham=prob.ham, L_coulomb=prob.Bc.shape[0], L_extra=Lx,
                   n_roots=n_roots or prob.n_roots,
                   level_shift_b=prob.level_shift_b if level_shift_b is None else level_shift_b,
                   class_mask=class_mask)

    def __del__(self):
        try:
            if self._h:
                load().e2_problem_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def workspace(self, device, solver=False, backward=False):
        """A 256-byte aligned uint8 CUDA tensor of the required size (cached);
        the reference solver and the adjoint need larger layouts, which
        contain the forward one."""
        import torch
        need = (self.backward_workspace_bytes if backward else
                self.solve_workspace_bytes if solver else self.workspace_bytes)
        if self._ws is None or self._ws.device != device or self._ws.numel() < need:
            self._ws = self._ws_raw = None   # free the smaller layout before taking the larger one
            raw = torch.empty(need + 256, dtype=torch.uint8, device=device)
            off = (-raw.data_ptr()) % 256
            self._ws_raw = raw
            self._ws = raw[off:off + need]
        return self._ws

    def release(self):
        """Drop the cached device workspace (the next call allocates again)."""
        self._ws = self._ws_raw = None

    def backward(self, h, B_c, c, B_x=None, w_x=None, lam=1.0, seed=None, want_h=True, want_c=True, want_B=False,
                 want_lambda=False, stream=None, E2_out=None):
        """Gradient of sum_m seed[m] E2_m: returns (g_h [n, n], g_c [roots, N_P],
        g_Bc [Lc, n, n], g_Bx [Lx, n, n], dE2/dlambda [1]) as CUDA tensors (None
        where not requested); complex gradients are dE/dRe + i dE/dIm, h and B
        Hermitian-projected.  E2_out (float64 CUDA [roots]), if given, receives
        the energies of the same pass."""
        import torch
        dev = c.device
        ws = self.workspace(dev, backward=True)
        seed = np.ascontiguousarray(np.ones(self.n_roots) if seed is None else seed, np.float64)
        gh = torch.empty(self.n, self.n, dtype=torch.complex128, device=dev) if want_h else None
        gc = torch.empty(self.n_roots, self.n_p, dtype=torch.complex128, device=dev) if want_c else None
        gbc = torch.empty(B_c.shape, dtype=torch.complex128, device=dev) if want_B else None
        gbx = torch.empty(B_x.shape, dtype=torch.complex128, device=dev) if (want_B and self.L_extra) else None
        dl = torch.zeros(1, dtype=torch.float64, device=dev) if want_lambda else None
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        ptr = lambda x: x.data_ptr() if x is not None else None
        _check(load().e2_backward(self._h, C.byref(inp), seed.ctypes.data_as(C.c_void_p), ws.data_ptr(), ws.numel(),
                                  C.c_void_p(s), ptr(gh), ptr(gc), ptr(gbc), ptr(gbx), ptr(dl), ptr(E2_out)))
        if want_B or want_lambda:
            return gh, gc, gbc, gbx, dl
        return gh, gc

    def value_and_grad(self, h, B_c, c, B_x=None, w_x=None, lam=1.0, seed=None, want_B=True, want_lambda=True,
                       stream=None):
        """E2 [roots] and the gradient of sum_m seed[m] E2_m from one pass
        (V formed once): returns (E2, g_h, g_c, g_Bc, g_Bx, dE2/dlambda)."""
        import torch
        E2 = torch.empty(self.n_roots, dtype=torch.float64, device=c.device)
        g = self.backward(h, B_c, c, B_x=B_x, w_x=w_x, lam=lam, seed=seed, want_B=want_B, want_lambda=want_lambda,
                          stream=stream, E2_out=E2)
        g = tuple(g) + (None,) * (5 - len(g))
        return (E2,) + g

    def reference_solve(self, h, B_c, X0, B_x=None, w_x=None, lam=1.0, tol=1e-10, max_iter=300, stream=None):
        """Lowest n_roots eigenvectors of P H P from start vectors X0 [roots, N_P]
        (complex128 CUDA).  Returns (c [roots, N_P] CUDA, E0 numpy, iterations)."""
        import torch
        dev = X0.device
        ws = self.workspace(dev, solver=True)
        c = torch.empty_like(X0)
        E0 = np.zeros(self.n_roots)
        it = C.c_int()
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), X0.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_reference_solve(self._h, C.byref(inp), tol, max_iter, ws.data_ptr(), ws.numel(),
                                         C.c_void_p(s), c.data_ptr(), E0.ctypes.data_as(C.c_void_p), C.byref(it)))
        return c, E0, int(it.value)

    def partials(self, root, cls):
        """Per-CTA partial sums of class cls (3h+p) for `root` from the last
        forward() (or value_and_grad()) as a float64 CUDA tensor view of the
        workspace, the row-tile count of a dense class (0 otherwise), and the
        column map of a class that uses column tiles (int32 CUDA view, list
        index per tile column, -1 = padding) or None."""
        import torch
        ptr, cnt, rt, cols = C.c_void_p(), C.c_int64(), C.c_int64(), C.c_void_p()
        _check(load().e2_partials(self._h, C.c_void_p(self._ws.data_ptr()), root, cls, C.byref(ptr), C.byref(cnt),
                                  C.byref(rt), C.byref(cols)))
        if cnt.value == 0:
            return torch.empty(0, dtype=torch.float64, device=self._ws.device), int(rt.value), None
        off = ptr.value - self._ws.data_ptr()
        part = self._ws[off:off + 8 * cnt.value].view(torch.float64)
        perm = None
        if cols.value:
            tiles, _, _ = self.class_tiles(cls)
            co = cols.value - self._ws.data_ptr()
            perm = self._ws[co:co + 4 * 64 * tiles].view(torch.int32)
        return part, int(rt.value), perm

    def status(self, stream=None, workspace=None):
        """Device status word of the last forward (or value_and_grad) on this
        problem's workspace: (code, flags, min_abs_D [roots, 9]) with code the
        e2_status it reports (0, E2_ERR_NONFINITE = 6 or E2_ERR_INTRUDER = 7),
        flags its bits (1: non-finite energy, 2: intruder denominator) and
        min_abs_D the smallest |E0 - H_KK| per root and class.  Synchronises."""
        import torch
        ws = self._ws if workspace is None else workspace
        flags = C.c_uint32()
        mind = np.zeros((self.n_roots, NCLASS))
        dev = ws.device if ws is not None else torch.device("cuda", torch.cuda.current_device())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        code = load().e2_query_status(self._h, C.c_void_p(ws.data_ptr()) if ws is not None else None, C.c_void_p(s),
                                      C.byref(flags), mind.ctypes.data_as(C.c_void_p))
        return int(code), int(flags.value), mind

    FAMILIES = {"t": 0, "t+": 1, "tu": 2, "t+u+": 3, "t+u": 4}

    def coupling_tables(self, family, h, B_c, c, B_x=None, w_x=None, lam=1.0, root=0, stream=None):
        """One coupling-tensor family of root `root` (e2_coupling_tables):
        returns (table [rows, n_A] complex128 CUDA, strings [n_A] int64 CUDA
        holding the uint64 bitsets)."""
        import torch
        L = load()
        fam = self.FAMILIES[family]
        rows, nA = C.c_int64(), C.c_int64()
        _check(L.e2_coupling_tables(self._h, None, None, 0, None, int(root), fam, None, None, C.byref(rows),
                                    C.byref(nA)))
        dev = c.device
        tab = torch.empty(int(rows.value), int(nA.value), dtype=torch.complex128, device=dev)
        strs = torch.empty(int(nA.value), dtype=torch.int64, device=dev)
        if nA.value == 0:
            return tab, strs
        ws = self.workspace(dev)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(L.e2_coupling_tables(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s), int(root), fam,
                                    C.c_void_p(tab.data_ptr()), C.c_void_p(strs.data_ptr()), None, None))
        return tab, strs

    def probe_couplings(self, cls, h, B_c, c, B_x=None, w_x=None, lam=1.0, root=0, tile_m=0, tile_n=0,
                        stream=None):
        """V and D of one tile of a dense class (64 x 64) or of a whole gather
        class ([rows, n_A]) from the class's FP64 kernel (e2_probe_couplings):
        returns (V complex128 CUDA, D float64 CUDA)."""
        import torch
        L = load()
        shape = (C.c_int64 * 2)()
        _check(L.e2_probe_couplings(self._h, None, None, 0, None, int(root), int(cls), 0, 0, None, None, shape))
        dev = c.device
        V = torch.zeros((shape[0], shape[1]), dtype=torch.complex128, device=dev)
        D = torch.zeros((shape[0], shape[1]), dtype=torch.float64, device=dev)
        ws = self.workspace(dev)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(L.e2_probe_couplings(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s), int(root),
                                    int(cls), int(tile_m), int(tile_n), C.c_void_p(V.data_ptr()),
                                    C.c_void_p(D.data_ptr()), None))
        return V, D

    DHIST = 18

    def denominator_histogram(self, h, B_c, c, B_x=None, w_x=None, lam=1.0, root=0, stream=None):
        """Counts of |E0 - H_KK| per class and decade (e2_denominator_histogram):
        int64 CUDA [9, 18]; bin 0 below 1e-12 Eh, bin k 10^(k-13)..10^(k-12),
        bin 17 the rest."""
        import torch
        dev = c.device
        hist = torch.zeros(NCLASS, self.DHIST, dtype=torch.int64, device=dev)
        ws = self.workspace(dev)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_denominator_histogram(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s),
                                               int(root), C.c_void_p(hist.data_ptr())))
        return hist

    def form_integrals(self, h, B_c, B_x=None, w_x=None, lam=1.0, c=None, stream=None):
        """The integral blocks of the classes from the factors alone
        (e2_form_integrals), in the cached workspace."""
        import torch
        dev = B_c.device
        ws = self.workspace(dev)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr() if c is not None else None)
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_form_integrals(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s)))

    def set_external_das(self, core_size=(), core_max_holes=(), virt_size=(), virt_max_particles=()):
        """Core / virtual DAS subspaces with per-subspace hole / particle limits
        (e2_set_external_das); empty sequences remove the limits.  Updates
        q_per_class."""
        cs = np.ascontiguousarray(core_size, np.int32)
        ch = np.ascontiguousarray(core_max_holes, np.int32)
        vs = np.ascontiguousarray(virt_size, np.int32)
        vp = np.ascontiguousarray(virt_max_particles, np.int32)
        _check(load().e2_set_external_das(self._h, len(cs), cs.ctypes.data_as(C.c_void_p),
                                          ch.ctypes.data_as(C.c_void_p), len(vs), vs.ctypes.data_as(C.c_void_p),
                                          vp.ctypes.data_as(C.c_void_p)))
        n_p = C.c_int64()
        q = np.zeros(NCLASS)
        _check(load().e2_problem_info(self._h, C.byref(n_p), q.ctypes.data_as(C.c_void_p)))
        self.q_per_class = q

    def set_shard(self, rank, n_ranks):
        """Take rank `rank`'s share of every class's units out of n_ranks
        (e2_set_shard; (0, 1) = unsharded)."""
        _check(load().e2_set_shard(self._h, int(rank), int(n_ranks)))

    def shard_units(self, cls):
        """(units of class cls, this rank's first, end)."""
        u, a, b = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().e2_shard_units(self._h, int(cls), C.byref(u), C.byref(a), C.byref(b)))
        return int(u.value), int(a.value), int(b.value)

    def shard_buffers(self):
        """(partials float64 CUDA view, smallest-|D| keys int64 CUDA view) of
        the workspace, for the ranks' collective."""
        import torch
        ws = self._ws
        p, n, k, nk = C.c_void_p(), C.c_int64(), C.c_void_p(), C.c_int64()
        _check(load().e2_shard_buffers(self._h, C.c_void_p(ws.data_ptr()), C.byref(p), C.byref(n), C.byref(k),
                                       C.byref(nk)))
        po, ko = p.value - ws.data_ptr(), k.value - ws.data_ptr()
        return (ws[po:po + 8 * n.value].view(torch.float64), ws[ko:ko + 8 * nk.value].view(torch.int64))

    def reduce(self, stream=None, out=None):
        """E2, E2_class, E0 from the partials in the workspace (after the
        ranks' sum): e2_reduce."""
        import torch
        dev = self._ws.device
        if out is None:
            out = (torch.empty(self.n_roots, dtype=torch.float64, device=dev),
                   torch.empty(self.n_roots, NCLASS, dtype=torch.float64, device=dev),
                   torch.empty(self.n_roots, dtype=torch.float64, device=dev))
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_reduce(self._h, C.c_void_p(self._ws.data_ptr()), self._ws.numel(), C.c_void_p(s),
                                C.c_void_p(out[0].data_ptr()), C.c_void_p(out[1].data_ptr()),
                                C.c_void_p(out[2].data_ptr())))
        return out

    def checkpointed_forward(self, path, h, B_c, c, B_x=None, w_x=None, lam=1.0, pieces=8, max_pieces=None,
                             tag=""):
        """E2 of a long run in `pieces` resumable parts (checkpoint / resume).
        Part k is shard k of `pieces` (e2_set_shard + e2_forward); as each
        completes, its partial slots and smallest-|D| keys are saved to
        `path`/piece_k.npz.  Parts already saved are skipped, so a killed run
        resumes where it stopped; `max_pieces` bounds the parts computed by
        this call.  When every part is saved: e2_prepare_roots, the parts'
        partials summed element-wise into the workspace (disjoint slots, so
        the sum is exact) and e2_reduce, giving E2, E2_class and E0 bitwise
        equal to the unsharded forward.  Returns (E2, E2_class, E0) then, else
        None.  `tag` names the inputs in the manifest: a directory holding
        parts of another problem or tag is refused."""
        import json
        import torch
        os.makedirs(path, exist_ok=True)
        ws = self.workspace(c.device)
        n_part = self.shard_buffers()[0].numel()
        meta = {"pieces": int(pieces), "partials": int(n_part), "roots": self.n_roots, "tag": str(tag),
                "q_per_class": [float(x) for x in self.q_per_class]}
        mpath = os.path.join(path, "manifest.json")
        if os.path.exists(mpath):
            if json.load(open(mpath)) != meta:
                raise E2Error(f"checkpoint directory {path} holds another run")
        else:
            json.dump(meta, open(mpath, "w"))
        kw = dict(B_x=B_x, w_x=w_x, lam=lam)
        done = 0
        try:
            for k in range(pieces):
                f = os.path.join(path, f"piece_{k}.npz")
                if os.path.exists(f):
                    continue
                if max_pieces is not None and done >= max_pieces:
                    return None
                self.set_shard(k, pieces)
                self.forward(h, B_c, c, **kw)
                part, keys = self.shard_buffers()
                tmp = f + ".tmp.npz"
                np.savez(tmp, part=part.cpu().numpy(), keys=keys.cpu().numpy())
                os.replace(tmp, f)
                done += 1
        finally:
            self.set_shard(0, 1)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(c.device).cuda_stream
        _check(load().e2_prepare_roots(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s)))
        part, keys = self.shard_buffers()
        part.zero_()
        keys.fill_(0x7FFFFFFFFFFFFFFF)
        for k in range(pieces):
            z = np.load(os.path.join(path, f"piece_{k}.npz"))
            part.add_(torch.from_numpy(z["part"]).to(part.device))
            torch.minimum(keys, torch.from_numpy(z["keys"]).to(keys.device), out=keys)
        return self.reduce()

    def sharded_forward(self, dist, h, B_c, c, B_x=None, w_x=None, lam=1.0, group=None):
        """E2 of the whole external space from this rank's share: e2_forward on
        the shard, the partials summed and the |D| keys minimised over the
        ranks of `group` (torch.distributed), then e2_reduce.  Bitwise equal
        to the unsharded forward for any number of ranks."""
        self.set_shard(dist.get_rank(group), dist.get_world_size(group))
        self.forward(h, B_c, c, B_x=B_x, w_x=w_x, lam=lam)
        part, keys = self.shard_buffers()
        dist.all_reduce(part, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(keys, op=dist.ReduceOp.MIN, group=group)
        return self.reduce()

    def class_tiles(self, cls):
        """(tiles, compacted rows, in use) of class cls's column tiles."""
        t, k, u = C.c_int64(), C.c_int64(), C.c_int()
        _check(load().e2_class_tiles(self._h, cls, C.byref(t), C.byref(k), C.byref(u)))
        return int(t.value), int(k.value), bool(u.value)

    def class_tiles_plan(self, cls):
        """Host copies (perm [tiles*64], tdesc [tiles, 4], klist [krows]) of
        class cls's column tiles."""
        tiles, krows, _ = self.class_tiles(cls)
        perm = np.zeros(tiles * 64, np.int32)
        tdesc = np.zeros((tiles, 4), np.int32)
        klist = np.zeros(max(krows, 1), np.int32)
        _check(load().e2_class_tiles_copy(self._h, cls, perm.ctypes.data_as(C.c_void_p),
                                          tdesc.ctypes.data_as(C.c_void_p), klist.ctypes.data_as(C.c_void_p)))
        return perm, tdesc, klist[:krows]

    def set_class_tiles(self, cls, on):
        _check(load().e2_set_class_tiles(self._h, cls, int(bool(on))))

    def set_contraction(self, cls, sliced):
        """Arithmetic of part of the path: True for the sliced bf16 tensor-pipe
        form with float-float epilogues (the default where available), False
        for FP64.  cls: a dense class (2, 5, 6, 7), 8 for class (2,2) (float-
        float elementwise kernel), -1 for the integral products of the setup,
        -2 for the products of the backward pass."""
        _check(load().e2_set_contraction(self._h, cls, 1 if sliced else 0))

    SLICEABLE = (2, 5, 6, 7, 8, -1, -2)

    def set_arithmetic(self, sliced):
        """The whole path in FP64 (sliced=False, the library's default) or, where
        the plan has it, in the emulated bf16-slice / float-float form
        (sliced=True); the other parts stay FP64."""
        for cls in self.SLICEABLE:
            if not sliced or self.contraction(cls)[1]:
                self.set_contraction(cls, bool(sliced))

    def arithmetic(self):
        """"fp64" when every part runs in FP64, else "sliced" (some part emulated)."""
        return "sliced" if any(self.contraction(cls)[0] for cls in self.SLICEABLE) else "fp64"

    def contraction(self, cls):
        """(sliced in use, sliced available) for cls as in set_contraction."""
        m, a = C.c_int(), C.c_int()
        _check(load().e2_contraction(self._h, cls, C.byref(m), C.byref(a)))
        return bool(m.value), bool(a.value)

    def set_adjoint_chunks(self, rows=0, core_pairs=0):
        """Run the adjoint in smaller chunks than planned (0 restores the plan)."""
        _check(load().e2_set_adjoint_chunks(self._h, int(rows), int(core_pairs)))

    def autotune(self, h, B_c, c, B_x=None, w_x=None, lam=1.0, stream=None):
        """Time plain against compacted columns per class and keep the faster;
        returns {class: (ms plain, ms compacted)} for the classes tried."""
        import torch
        ws = self.workspace(c.device)
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(c.device).cuda_stream if stream is None else stream
        ms = (C.c_float * (2 * NCLASS))()
        _check(load().e2_autotune(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s), ms))
        return {k: (ms[2 * k], ms[2 * k + 1]) for k in range(NCLASS) if ms[2 * k] > 0}

    def tuning_save(self, path):
        """Append this problem's column-tile choices to the tuning cache file."""
        _check(load().e2_tuning_save(self._h, os.fsencode(path)))

    def tuning_load(self, path):
        """Apply the cached choices for this problem's shape; False when the
        file holds none (the plan's defaults stay)."""
        st = load().e2_tuning_load(self._h, os.fsencode(path))
        if st == 3:
            return False
        _check(st)
        return True

    def launch_count(self):
        """Kernels enqueued by the last forward()."""
        n = C.c_int64()
        _check(load().e2_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def set_events(self, pairs):
        """Point the class-kernel hooks at (start, end) torch.cuda.Event pairs
        (already recorded once) or switch them off with None; no sync."""
        if pairs is None:
            _check(load().e2_profile_events(self._h, None))
            return
        arr = (C.c_void_p * (2 * NCLASS))()
        for k, (a, b) in enumerate(pairs):
            arr[2 * k] = a.cuda_event
            arr[2 * k + 1] = b.cuda_event
        self._event_arr = arr
        _check(load().e2_profile_events(self._h, arr))

    def profile(self, on=True):
        """Record CUDA events around each class kernel of root 0 in forward();
        returns the list of (start, end) torch.cuda.Event pairs per class."""
        import torch
        if not on:
            _check(load().e2_profile_events(self._h, None))
            self._events = None
            return None
        self._events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                        for _ in range(NCLASS)]
        arr = (C.c_void_p * (2 * NCLASS))()
        for k, (a, b) in enumerate(self._events):
            a.record()  # materialise the handles
            b.record()
            arr[2 * k] = a.cuda_event
            arr[2 * k + 1] = b.cuda_event
        torch.cuda.synchronize()
        _check(load().e2_profile_events(self._h, arr))
        return self._events

    def forward(self, h, B_c, c, B_x=None, w_x=None, lam=1.0, stream=None, workspace=None, out=None):
        """E2 per root.  Tensors: complex128 CUDA, contiguous.  Returns
        (E2 [roots], E2_class [roots, 9], E0 [roots]) as float64 CUDA tensors."""
        import torch
        dev = c.device
        for t in (h, B_c, c) + ((B_x,) if self.L_extra else ()):
            if t.dtype != torch.complex128 or not t.is_contiguous() or t.device != dev:
                raise E2Error("inputs must be contiguous complex128 tensors on one CUDA device")
        if c.numel() != self.n_roots * self.n_p:
            raise E2Error(f"c must hold n_roots*N_P = {self.n_roots * self.n_p} coefficients")
        ws = self.workspace(dev) if workspace is None else workspace
        if out is None:
            out = (torch.empty(self.n_roots, dtype=torch.float64, device=dev),
                   torch.empty(self.n_roots, NCLASS, dtype=torch.float64, device=dev),
                   torch.empty(self.n_roots, dtype=torch.float64, device=dev))
        E2, E2c, E0 = out
        inp = _Inputs(h.data_ptr(), B_c.data_ptr(), B_x.data_ptr() if self.L_extra else None,
                      w_x.data_ptr() if self.L_extra else None, float(lam), c.data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_forward(self._h, C.byref(inp), ws.data_ptr(), ws.numel(), C.c_void_p(s), E2.data_ptr(),
                                 E2c.data_ptr(), E0.data_ptr()))
        return E2, E2c, E0


class E2Batch:
    """Several planned problems whose classes (every job, root and class) are
    evaluated by one persistent launch (e2_batch_*), or one per group of
    roots_per_launch roots.  forward() enqueues kernels and device copies
    only, so it can be captured in a CUDA graph after prepare()."""

    def __init__(self, plans, roots_per_launch=0):
        L = load()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h for p in self.plans])
        h = C.c_void_p()
        _check(L.e2_batch_create(arr, len(self.plans), C.byref(h)))
        self._h = h
        if roots_per_launch:
            _check(L.e2_batch_set_roots_per_launch(self._h, int(roots_per_launch)))
        ws = C.c_size_t()
        _check(L.e2_batch_workspace_size(self._h, C.byref(ws)))
        self.workspace_bytes = int(ws.value)
        self._ws = None

    def __del__(self):
        try:
            if self._h:
                load().e2_batch_destroy(self._h)
                self._h = None
        except Exception:
            pass

    @staticmethod
    def plan_batches(plans, budget_bytes):
        """Split planned jobs into batches whose workspaces fit budget_bytes
        (host only; the sizes come from e2_batch_workspace_size).  Jobs are
        taken in order; each batch gets the most jobs that fit with one table
        slot per job (roots_per_launch = 1), then the largest roots_per_launch
        that still fits (0 when every root fits in one launch).  Returns
        [(jobs, roots_per_launch)]; raises E2Error if one job alone does not
        fit."""
        def size(group, k):
            return E2Batch(group, roots_per_launch=k).workspace_bytes

        out, i = [], 0
        plans = list(plans)
        while i < len(plans):
            j = i + 1
            if size(plans[i:j], 1) > budget_bytes:
                raise E2Error("a job does not fit the budget even with one coupling-table slot")
            while j < len(plans) and size(plans[i:j + 1], 1) <= budget_bytes:
                j += 1
            group = plans[i:j]
            roots = max(p.n_roots for p in group)
            k = 0 if size(group, 0) <= budget_bytes else max(
                kk for kk in range(1, roots + 1) if size(group, kk) <= budget_bytes)
            out.append((group, k))
            i = j
        return out

    def prepare(self, device, stream=None):
        import torch
        raw = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=device)
        off = (-raw.data_ptr()) % 256
        self._ws_raw = raw
        self._ws = raw[off:off + self.workspace_bytes]
        s = torch.cuda.current_stream(device).cuda_stream if stream is None else stream
        _check(load().e2_batch_prepare(self._h, self._ws.data_ptr(), self._ws.numel(), C.c_void_p(s)))
        self.outputs = [(torch.empty(p.n_roots, dtype=torch.float64, device=device),
                         torch.empty(p.n_roots, NCLASS, dtype=torch.float64, device=device)) for p in self.plans]

    def forward(self, inputs, stream=None):
        """inputs: one dict per job (as from device_inputs).  Returns the
        per-job (E2, E2_class) tensors (reused between calls)."""
        import torch
        dev = self._ws.device
        self._keep = []
        arr = (_Inputs * len(self.plans))()
        for k, (p, t) in enumerate(zip(self.plans, inputs)):
            arr[k] = _Inputs(t["h"].data_ptr(), t["B_c"].data_ptr(), t["B_x"].data_ptr() if p.L_extra else None,
                             t["w_x"].data_ptr() if p.L_extra else None, float(t["lam"]), t["c"].data_ptr())
        e2p = (C.c_void_p * len(self.plans))(*[o[0].data_ptr() for o in self.outputs])
        e2c = (C.c_void_p * len(self.plans))(*[o[1].data_ptr() for o in self.outputs])
        self._keep = [arr, e2p, e2c]
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(load().e2_batch_forward(self._h, C.cast(arr, C.c_void_p), self._ws.data_ptr(), self._ws.numel(),
                                       C.c_void_p(s), C.cast(e2p, C.c_void_p), C.cast(e2c, C.c_void_p)))
        return self.outputs

    def launch_count(self):
        n = C.c_int64()
        _check(load().e2_batch_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def backward(self, inputs, seeds=None, want_B=True, stream=None):
        """Every job's adjoint (e2_batch_backward): returns per job (E2, g_h,
        g_c, g_Bc, g_Bx, dE2/dlambda) as CUDA tensors."""
        import torch
        L = load()
        dev = inputs[0]["c"].device
        need = C.c_size_t()
        _check(L.e2_batch_backward_workspace_size(self._h, C.byref(need)))
        raw = torch.empty(need.value + 256, dtype=torch.uint8, device=dev)
        off = (-raw.data_ptr()) % 256
        ws = raw[off:off + need.value]
        nj = len(self.plans)
        arr = (_Inputs * nj)()
        seeds = [np.ones(p.n_roots) if seeds is None else np.ascontiguousarray(seeds[j], np.float64)
                 for j, p in enumerate(self.plans)]
        seeds = [np.ascontiguousarray(x, np.float64) for x in seeds]
        sp = (C.c_void_p * nj)(*[x.ctypes.data for x in seeds])
        outs = []
        for k, (p, t) in enumerate(zip(self.plans, inputs)):
            arr[k] = _Inputs(t["h"].data_ptr(), t["B_c"].data_ptr(), t["B_x"].data_ptr() if p.L_extra else None,
                             t["w_x"].data_ptr() if p.L_extra else None, float(t["lam"]), t["c"].data_ptr())
            outs.append((torch.empty(p.n_roots, dtype=torch.float64, device=dev),
                         torch.empty(p.n, p.n, dtype=torch.complex128, device=dev),
                         torch.empty(p.n_roots, p.n_p, dtype=torch.complex128, device=dev),
                         torch.empty(t["B_c"].shape, dtype=torch.complex128, device=dev) if want_B else None,
                         torch.empty(t["B_x"].shape, dtype=torch.complex128, device=dev)
                         if (want_B and p.L_extra) else None,
                         torch.zeros(1, dtype=torch.float64, device=dev)))
        ptrs = lambda i: (C.c_void_p * nj)(*[o[i].data_ptr() if o[i] is not None else None for o in outs])
        s = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        _check(L.e2_batch_backward(self._h, C.cast(arr, C.c_void_p), C.cast(sp, C.c_void_p), ws.data_ptr(),
                                   ws.numel(), C.c_void_p(s), ptrs(1), ptrs(2), ptrs(3), ptrs(4), ptrs(5), ptrs(0)))
        return outs


def fp64_peak(device="cuda"):
    """Measured FP64 tensor-pipe (mma.sync f64) and FP64 FMA TFLOP/s of the device."""
    import torch
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    buf = torch.empty(8 * 256 * 8 * sms, dtype=torch.uint8, device=device)
    a, b = C.c_double(), C.c_double()
    _check(load().e2_fp64_peak(buf.data_ptr(), buf.numel(), C.c_void_p(torch.cuda.current_stream(device).cuda_stream),
                               C.byref(a), C.byref(b)))
    return a.value, b.value


def device_inputs(prob, c, device="cuda"):
    """Copy an ``e2_inputs.Problem`` and coefficients c [roots, N_P] to the device."""
    import torch
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(device=device, dtype=dt)
    h = t(prob.h, torch.complex128)
    Bc = t(prob.Bc, torch.complex128)
    Bx = t(prob.Bx, torch.complex128) if prob.ham != "DC" and prob.Bx.shape[0] else None
    wx = t(prob.wx, torch.float64) if Bx is not None else None
    cc = t(np.atleast_2d(c), torch.complex128)
    return dict(h=h, B_c=Bc, B_x=Bx, w_x=wx, c=cc, lam=prob.lam)
