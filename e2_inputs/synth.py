"""Synthetic problem recipe (numbers and layout only).

Recipe, per configuration (see the module docstring for the spinor order):

* spinor energies eps: core values geometric between the stated ends, active
  values linear in [-1, 0], virtual values log-spaced between the stated ends;
  each value is used by both members of a Kramers pair.
* one-body h = diag(eps) + a Hermitian off-diagonal part whose upper triangle is
  0.01 (x + i y) exp(-|p-q|/8), x, y ~ N(0, 1).
* factor sets B^L (Hermitian n x n, one per L): upper triangle
  0.1 (x + i y) exp(-|p-q|/8), diagonal 0.1 x, x, y ~ N(0, 1).  The Coulomb set
  has weight 1 per factor; the Gaunt (DCG) or Breit (DCB) set has weight
  s * sigma_L with sigma_L a seeded Rademacher sign and s the stated scale; the
  call multiplies the extra set by lambda (1 by default).
* start vectors X0 [n_roots][N_P] with complex N(0, 1) entries for the
  reference-state eigen-solve.

With ``time_reversal=True`` the one-body matrix and the Coulomb factors are
built Kramers-symmetric (2x2 pair blocks [[a, b], [-b*, a*]]) and the extra
factors Kramers-antisymmetric ([[a, b], [b*, -a*]]); the two-electron operator
is then time-reversal invariant.
"""
from __future__ import annotations

import dataclasses
from math import comb
from typing import List, Optional

import numpy as np

HAMILTONIANS = ("DC", "DCG", "DCB")

# Stream ids for numpy.random.default_rng([config_id, stream, ...]).
_S_H, _S_BC, _S_BX, _S_SIGN, _S_X0 = 1, 2, 3, 4, 5


@dataclasses.dataclass
class Problem:
    name: str
    n_core: int
    n_act: int
    n_virt: int
    n_elec: int                  # active electrons of the reference space
    das_size: List[int]          # sizes of the active subspaces (sum = n_act)
    das_min: List[int]           # minimum electrons per subspace in P
    das_max: List[int]           # maximum electrons per subspace in P
    ham: str                     # "DC", "DCG" or "DCB"
    eps: np.ndarray              # [n] float64
    h: np.ndarray                # [n, n] complex128, Hermitian
    Bc: np.ndarray               # [Lc, n, n] complex128, Hermitian per factor
    Bx: np.ndarray               # [Lx, n, n] complex128 (Gaunt or Breit set)
    wx: np.ndarray               # [Lx] float64 signed weights of the extra set
    lam: float                   # multiplier of the extra set
    n_roots: int
    frozen: np.ndarray           # [n] uint8, 1 = frozen spinor
    X0: np.ndarray               # [n_roots, N_P] complex128 start vectors
    level_shift_b: float = 0.0

    @property
    def n(self) -> int:
        return self.n_core + self.n_act + self.n_virt

    @property
    def n_p(self) -> int:
        return n_p_space(self.das_size, self.das_min, self.das_max, self.n_elec)

    def factors(self):
        """All factor sets with their weights: ((pq|rs) = sum_L w_L B_pq B_rs)."""
        if self.Bx.shape[0] == 0 or self.ham == "DC":
            return self.Bc, np.ones(self.Bc.shape[0])
        B = np.concatenate([self.Bc, self.Bx], axis=0)
        w = np.concatenate([np.ones(self.Bc.shape[0]), self.lam * self.wx])
        return B, w


def pattern_count(das_size, pattern):
    out = 1
    for s, k in zip(das_size, pattern):
        out *= comb(s, k)
    return out


def das_patterns(das_size, das_min, das_max, n_elec):
    """Occupation patterns (n_1..n_k) with min <= n_s <= max and sum n_elec,
    lexicographic with n_1 most significant (the address order of c)."""
    out = []

    def rec(s, left, cur):
        if s == len(das_size):
            if left == 0:
                out.append(tuple(cur))
            return
        for k in range(das_min[s], min(das_max[s], das_size[s]) + 1):
            if k <= left:
                rec(s + 1, left - k, cur + [k])

    rec(0, n_elec, [])
    return out


def n_p_space(das_size, das_min, das_max, n_elec) -> int:
    return sum(pattern_count(das_size, p) for p in das_patterns(das_size, das_min, das_max, n_elec))


def _eps(n_core, n_act, n_virt, core_ends, virt_ends):
    cp, ap, vp = n_core // 2, n_act // 2, n_virt // 2
    core = -np.geomspace(-core_ends[0], -core_ends[1], cp) if cp else np.zeros(0)
    act = np.linspace(-1.0, 0.0, ap) if ap > 1 else np.full(ap, -0.5)
    virt = np.geomspace(virt_ends[0], virt_ends[1], vp) if vp else np.zeros(0)
    return np.repeat(np.concatenate([core, act, virt]), 2)


def _decay(n):
    d = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    return np.exp(-d / 8.0)


def _hermitian(rng, n, scale, dec):
    x = scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * dec
    x = np.triu(x, 1)
    return x + x.conj().T + np.diag(scale * rng.standard_normal(n))


def _kramers(rng, n, scale, dec, odd):
    """Hermitian matrix with Kramers pair structure (even: [[a,b],[-b*,a*]],
    odd: [[a,b],[b*,-a*]]), entries scaled like _hermitian."""
    m = n // 2
    M = np.zeros((n, n), complex)
    for k in range(m):
        for l in range(k, m):
            f = scale * dec[2 * k, 2 * l]
            if k == l:
                a = f * rng.standard_normal()
                b = f * (rng.standard_normal() + 1j * rng.standard_normal()) if odd else 0.0
            else:
                a = f * (rng.standard_normal() + 1j * rng.standard_normal())
                b = f * (rng.standard_normal() + 1j * rng.standard_normal())
            blk = np.array([[a, b], [np.conj(b), -np.conj(a)]]) if odd else \
                np.array([[a, b], [-np.conj(b), np.conj(a)]])
            M[2 * k:2 * k + 2, 2 * l:2 * l + 2] = blk
            if k != l:
                M[2 * l:2 * l + 2, 2 * k:2 * k + 2] = blk.conj().T
    return M


def tiny_problem(n_core, n_act, n_virt, n_elec, *, Lc=6, Lx=0, ham="DC", x_scale=1e-2,
                 das_size=None, das_min=None, das_max=None, core_ends=(-20.0, -2.0),
                 virt_ends=(0.1, 50.0), n_roots=1, n_frozen_core=0, n_frozen_virt=0,
                 seed=0, time_reversal=False, h_offdiag=0.01, b_scale=0.1, lam=1.0,
                 level_shift_b=0.0, name=None) -> Problem:
    """Build a problem from sizes.  All sizes are spinor counts (even)."""
    assert ham in HAMILTONIANS
    if ham == "DC":
        Lx = 0
    n = n_core + n_act + n_virt
    if das_size is None:
        das_size, das_min, das_max = [n_act], [n_elec], [n_elec]
    assert sum(das_size) == n_act
    eps = _eps(n_core, n_act, n_virt, core_ends, virt_ends)
    dec = _decay(n)
    rng = np.random.default_rng([seed, _S_H])
    if time_reversal:
        h = np.diag(eps).astype(complex) + _kramers(rng, n, h_offdiag, dec, odd=False) * (1 - np.eye(n))
    else:
        off = h_offdiag * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) * dec
        off = np.triu(off, 1)
        h = np.diag(eps).astype(complex) + off + off.conj().T
    Bc = np.empty((Lc, n, n), complex)
    for l in range(Lc):
        r = np.random.default_rng([seed, _S_BC, l])
        Bc[l] = _kramers(r, n, b_scale, dec, odd=False) if time_reversal else _hermitian(r, n, b_scale, dec)
    xs = _S_BX * 10 + HAMILTONIANS.index(ham)   # independent Gaunt / Breit draws
    Bx = np.empty((Lx, n, n), complex)
    for l in range(Lx):
        r = np.random.default_rng([seed, xs, l])
        Bx[l] = _kramers(r, n, b_scale, dec, odd=True) if time_reversal else _hermitian(r, n, b_scale, dec)
    sgn = np.random.default_rng([seed, _S_SIGN, xs]).integers(0, 2, Lx) * 2 - 1
    wx = x_scale * sgn.astype(float)
    frozen = np.zeros(n, np.uint8)
    frozen[:n_frozen_core] = 1
    if n_frozen_virt:
        frozen[n - n_frozen_virt:] = 1
    n_p = n_p_space(das_size, das_min, das_max, n_elec)
    r = np.random.default_rng([seed, _S_X0])
    X0 = r.standard_normal((n_roots, n_p)) + 1j * r.standard_normal((n_roots, n_p))
    return Problem(name=name or f"tiny_{n_core}_{n_act}_{n_virt}_{n_elec}", n_core=n_core, n_act=n_act,
                   n_virt=n_virt, n_elec=n_elec, das_size=list(das_size), das_min=list(das_min),
                   das_max=list(das_max), ham=ham, eps=eps, h=h, Bc=Bc, Bx=Bx, wx=wx, lam=lam,
                   n_roots=n_roots, frozen=frozen, X0=X0, level_shift_b=level_shift_b)


# The five workload shapes (Ne- to Xe-shaped).  Sizes are spinors.
CONFIGS = {
    # plain DC, CAS(6e,12), 924 reference determinants
    "dc_small": dict(n_core=4, n_act=12, n_virt=40, n_elec=6, Lc=60, Lx=0, ham="DC",
                 core_ends=(-20.0, -2.0), virt_ends=(0.1, 50.0), seed=1),
    # Ne-shaped DCG, CAS(8e,16), 12870 reference determinants
    "ne_dcg": dict(n_core=2, n_act=16, n_virt=200, n_elec=8, Lc=400, Lx=200, ham="DCG", x_scale=1e-3,
                 core_ends=(-33.0, -33.0), virt_ends=(0.2, 200.0), seed=2),
    # Ar-shaped DCB with three active subspaces of 8 (RAS-like 8/2/0 nominal)
    "ar_dcb_das": dict(n_core=8, n_act=24, n_virt=400, n_elec=10, Lc=600, Lx=300, ham="DCB", x_scale=2e-3,
                 das_size=[8, 8, 8], das_min=[6, 0, 0], das_max=[8, 8, 2],
                 core_ends=(-119.0, -9.5), virt_ends=(0.1, 200.0), seed=3),
    # Kr-shaped, CAS(8e,24), 4 roots; the batch varies Hamiltonian and frozen cutoffs
    "kr_dcb": dict(n_core=16, n_act=24, n_virt=600, n_elec=8, Lc=900, Lx=450, ham="DCB", x_scale=3e-3,
                 core_ends=(-520.0, -3.0), virt_ends=(0.1, 400.0), n_roots=4, seed=4),
    # Xe-shaped, CAS(8e,24), DCB
    "xe_dcb": dict(n_core=46, n_act=24, n_virt=1000, n_elec=8, Lc=1400, Lx=700, ham="DCB", x_scale=4e-3,
                 core_ends=(-1280.0, -2.5), virt_ends=(0.1, 800.0), seed=5),
}


def make_problem(name: str, **overrides) -> Problem:
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    return tiny_problem(name=name, **kw)
