"""ctypes front end of the C oracle (test infrastructure only).

Functions and the passages they follow:

* ``Oracle.e0``            -- E0_m = <Psi_m|H|Psi_m> / <Psi_m|Psi_m> (Sec. 2.3)
* ``Oracle.hpp``           -- P H P as a sparse matrix (Eq. zeroh, first term)
* ``Oracle.ground_state``  -- lowest eigenvectors of P H P, the reference states
                              (Sec. 2.3; CASCI reference, Sec. 2.2)
* ``Oracle.e2``            -- E2 per root and class (Eq. pt2, Eq. pt2en,
                              level shift of Sec. 2.6)
* ``Oracle.couplings``     -- V_K = <K|H|Psi> and E0 - H_KK for listed K
* ``Oracle.count_q``       -- size of Q per class (Sec. 2.3, Table 3)
* ``Oracle.hmat``          -- generic <K|H|L> between two determinants
* ``Oracle.set_external_das`` -- core / virtual DAS subspaces with hole /
                              particle limits restricting Q (Sec. 2.4, Fig. 1)
* ``Oracle.dtable``        -- coupling tensors D^x_A = <A|x|Psi> of listed
                              active strings by generic operator algebra
                              (Sec. 2.4, Eq. sumsigma: the <K|E_pq|L> C_L
                              factors restricted to the active space)

Class id = 3 * (core holes) + (virtual particles); class 0 is the pure
active rearrangement class that only a DAS partition has.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "e2_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
NCLASS = 9


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 + OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-Wall",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [("n_core", C.c_int), ("n_act", C.c_int), ("n_virt", C.c_int), ("n_elec", C.c_int),
                ("n_das", C.c_int), ("das_size", C.POINTER(C.c_int)), ("das_min", C.POINTER(C.c_int)),
                ("das_max", C.POINTER(C.c_int)), ("frozen", C.POINTER(C.c_ubyte)),
                ("h", C.POINTER(C.c_double)), ("L", C.c_int), ("B", C.POINTER(C.c_double)),
                ("w", C.POINTER(C.c_double)), ("level_shift_b", C.c_double),
                ("use_eri_cache", C.c_int), ("n_threads", C.c_int)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.oracle_create.restype = C.c_void_p
        L.oracle_create.argtypes = [C.POINTER(_Desc)]
        L.oracle_destroy.argtypes = [C.c_void_p]
        L.oracle_np.restype = C.c_int64
        L.oracle_np.argtypes = [C.c_void_p]
        L.oracle_set_c.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
        L.oracle_e0.argtypes = [C.c_void_p, C.c_void_p]
        L.oracle_hpp_coo.restype = C.c_int64
        L.oracle_hpp_coo.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.oracle_e2.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_couplings.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_count_q.argtypes = [C.c_void_p, C.c_void_p]
        L.oracle_hmat.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_maxw.restype = C.c_int
        L.oracle_eri.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]
        L.oracle_grad.argtypes = [C.c_void_p] + [C.c_void_p] * 6
        L.oracle_dtable.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p, C.c_void_p]
        L.oracle_set_external_das.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                              C.c_void_p]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """Oracle bound to one problem (an ``e2_inputs.Problem``)."""

    def __init__(self, prob, use_eri_cache=None, n_threads=0, level_shift_b=None):
        L = _load()
        self.prob = prob
        B, w = prob.factors()
        self._B = np.ascontiguousarray(B, dtype=np.complex128)
        self._w = np.ascontiguousarray(w, dtype=np.float64)
        self._h = np.ascontiguousarray(prob.h, dtype=np.complex128)
        self._frozen = np.ascontiguousarray(prob.frozen, dtype=np.uint8)
        self._ds = np.ascontiguousarray(prob.das_size, dtype=np.int32)
        self._dmin = np.ascontiguousarray(prob.das_min, dtype=np.int32)
        self._dmax = np.ascontiguousarray(prob.das_max, dtype=np.int32)
        n = prob.n
        if use_eri_cache is None:
            use_eri_cache = n <= 96
        b = prob.level_shift_b if level_shift_b is None else level_shift_b
        d = _Desc(prob.n_core, prob.n_act, prob.n_virt, prob.n_elec, len(prob.das_size),
                  self._ds.ctypes.data_as(C.POINTER(C.c_int)), self._dmin.ctypes.data_as(C.POINTER(C.c_int)),
                  self._dmax.ctypes.data_as(C.POINTER(C.c_int)),
                  self._frozen.ctypes.data_as(C.POINTER(C.c_ubyte)),
                  self._h.ctypes.data_as(C.POINTER(C.c_double)), self._B.shape[0],
                  self._B.ctypes.data_as(C.POINTER(C.c_double)), self._w.ctypes.data_as(C.POINTER(C.c_double)),
                  float(b), int(bool(use_eri_cache)), int(n_threads))
        self._h_ptr = L.oracle_create(C.byref(d))
        self._L = L
        self.n_p = int(L.oracle_np(self._h_ptr))
        self.n_roots = 0
        self.c = None

    def __del__(self):
        try:
            if self._h_ptr:
                self._L.oracle_destroy(self._h_ptr)
                self._h_ptr = None
        except Exception:
            pass

    # -- reference state -------------------------------------------------
    def set_c(self, c):
        c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.complex128)
        assert c.shape[1] == self.n_p
        self.c = c
        self.n_roots = c.shape[0]
        self._L.oracle_set_c(self._h_ptr, _ptr(c), self.n_roots)

    def hpp(self):
        import scipy.sparse as sp
        nnz = int(self._L.oracle_hpp_coo(self._h_ptr, None, None, None, 0))
        rows = np.empty(nnz, np.int64)
        cols = np.empty(nnz, np.int64)
        vals = np.empty(nnz, np.complex128)
        got = int(self._L.oracle_hpp_coo(self._h_ptr, _ptr(rows), _ptr(cols), _ptr(vals), nnz))
        assert got == nnz
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_p, self.n_p))

    def ground_state(self, n_roots=None, X0=None, tol=1e-12):
        """Lowest n_roots eigenvectors of P H P; each vector's largest-modulus
        entry is made real positive.  Sets c and returns (c, eigenvalues)."""
        n_roots = n_roots or self.prob.n_roots
        H = self.hpp()
        if self.n_p <= 3000:
            w, V = np.linalg.eigh(H.toarray())
            w, V = w[:n_roots], V[:, :n_roots]
        else:
            import scipy.sparse.linalg as sla
            v0 = None if X0 is None else np.asarray(X0)[0]
            w, V = sla.eigsh(H, k=n_roots, which="SA", v0=v0, tol=tol)
            o = np.argsort(w)
            w, V = w[o], V[:, o]
        c = V.T.copy()
        for m in range(n_roots):
            k = int(np.argmax(np.abs(c[m])))
            c[m] *= np.conj(c[m, k]) / abs(c[m, k])
            c[m] /= np.linalg.norm(c[m])
        self.set_c(c)
        return c, w

    # -- energies --------------------------------------------------------
    def e0(self):
        out = np.zeros(self.n_roots)
        self._L.oracle_e0(self._h_ptr, _ptr(out))
        return out

    def e2(self, E0=None):
        """Returns (E2[root], E2[root][class], couplings[class])."""
        if E0 is None:
            E0 = self.e0()
        E0 = np.ascontiguousarray(E0, dtype=np.float64)
        ec = np.zeros((self.n_roots, NCLASS))
        nc = np.zeros(NCLASS, np.int64)
        self._L.oracle_e2(self._h_ptr, _ptr(E0), _ptr(ec), _ptr(nc))
        return ec.sum(axis=1), ec, nc

    def couplings(self, E0, nh, holes, npart, parts, act):
        """V_K [nK][root] complex and D_K = E0 - H_KK [nK][root]."""
        nK = len(nh)
        nh = np.ascontiguousarray(nh, np.int32)
        npart = np.ascontiguousarray(npart, np.int32)
        holes = np.ascontiguousarray(np.reshape(holes, (nK, 2)), np.int32)
        parts = np.ascontiguousarray(np.reshape(parts, (nK, 2)), np.int32)
        act = np.ascontiguousarray(act, np.uint64)
        E0 = np.ascontiguousarray(E0, np.float64)
        V = np.zeros((nK, self.n_roots), np.complex128)
        D = np.zeros((nK, self.n_roots))
        self._L.oracle_couplings(self._h_ptr, _ptr(E0), nK, _ptr(nh), _ptr(holes), _ptr(npart), _ptr(parts),
                                 _ptr(act), _ptr(V), _ptr(D))
        return V, D

    def grad(self, E0=None, seed=None):
        """Gradient of sum_m seed[m] E2_m: returns (gh [n,n], gB [L,n,n] in the
        factor order of Problem.factors(), gw [L], gc [roots, N_P]); complex
        gradients are dE/dRe + i dE/dIm, Hermitian-projected for h and B."""
        if E0 is None:
            E0 = self.e0()
        E0 = np.ascontiguousarray(E0, np.float64)
        seed = np.ascontiguousarray(np.ones(self.n_roots) if seed is None else seed, np.float64)
        n, L = self.prob.n, self._B.shape[0]
        gh = np.zeros((n, n), np.complex128)
        gB = np.zeros((L, n, n), np.complex128)
        gw = np.zeros(L)
        gc = np.zeros((self.n_roots, self.n_p), np.complex128)
        self._L.oracle_grad(self._h_ptr, _ptr(E0), _ptr(seed), _ptr(gh), _ptr(gB), _ptr(gw), _ptr(gc))
        return gh, gB, gw, gc

    def set_external_das(self, core_size=(), core_max_holes=(), virt_size=(), virt_max_particles=()):
        """DAS subspaces of the core / virtual spinors (consecutive blocks) with
        per-subspace limits on holes / particles (Sec. 2.4, Fig. 1): Q keeps
        the determinants within every limit."""
        arrs = [np.ascontiguousarray(x, np.int32) for x in (core_size, core_max_holes, virt_size,
                                                              virt_max_particles)]
        self._xdas = arrs
        self._L.oracle_set_external_das(self._h_ptr, len(arrs[0]), _ptr(arrs[0]), _ptr(arrs[1]), len(arrs[2]),
                                        _ptr(arrs[2]), _ptr(arrs[3]))

    FAMILIES = {"t": 0, "t+": 1, "tu": 2, "t+u+": 3, "t+u": 4}

    def dtable(self, family, strings, root=0):
        """D^x_A for the active strings A (active-local bitsets) of one family:
        "t" <A|a_t|Psi>, "t+" <A|a+_t|Psi>, "tu" <A|a_u a_t|Psi> (t<u, row
        u(u-1)/2 + t), "t+u+" <A|a+_t a+_u|Psi> (t<u, same rows), "t+u" row 0
        c_A and row 1 + t n_act + u <A|a+_t a_u|Psi>.  Returns [rows, nA]
        complex128."""
        fam = self.FAMILIES[family]
        na = self.prob.n_act
        rows = na if fam <= 1 else na * (na - 1) // 2 if fam <= 3 else 1 + na * na
        A = np.ascontiguousarray(strings, np.uint64)
        out = np.zeros((rows, len(A)), np.complex128)
        self._L.oracle_dtable(self._h_ptr, fam, int(root), len(A), _ptr(A), _ptr(out))
        return out

    def count_q(self):
        out = np.zeros(NCLASS)
        self._L.oracle_count_q(self._h_ptr, _ptr(out))
        return out

    def eri(self, p, q, r, s):
        """(pq|rs) as the oracle evaluates it."""
        out = np.zeros(2)
        self._L.oracle_eri(self._h_ptr, p, q, r, s, _ptr(out))
        return complex(out[0], out[1])

    def hmat(self, K_occ, L_occ):
        """<K|H|L> for two determinants given as lists of occupied spinors."""
        W = self._L.oracle_maxw()
        kb = np.zeros(W, np.uint64)
        lb = np.zeros(W, np.uint64)
        for p in K_occ:
            kb[p // 64] |= np.uint64(1) << np.uint64(p % 64)
        for p in L_occ:
            lb[p // 64] |= np.uint64(1) << np.uint64(p % 64)
        out = np.zeros(2)
        self._L.oracle_hmat(self._h_ptr, _ptr(kb), _ptr(lb), _ptr(out))
        return complex(out[0], out[1])
