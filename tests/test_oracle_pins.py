"""Pins of the oracle against results fixed by the paper and by mathematics.

Each test ties the oracle to something other than itself: a brute-force
Jordan-Wigner Fock-space matrix, the paper's printed determinant counts
(Table 3), the textbook single-determinant Epstein-Nesbet formula, exact
symmetries (Hermiticity, time reversal, spinor phase gauge), and limits
(level shift b -> 0, frozen spinors = partial sums).
"""
import os
from itertools import combinations
from math import comb

import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from oracle import Oracle
from jw_fock import brute_e2, integrals, fock_hamiltonian, p_address

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _ground(prob, n_roots=None):
    o = Oracle(prob)
    c, w = o.ground_state(n_roots or prob.n_roots)
    return o, c, w


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("case", [
    dict(n_core=2, n_act=4, n_virt=4, n_elec=2, Lc=4, Lx=3, ham="DCB", x_scale=0.05, n_roots=2, seed=3),
    dict(n_core=4, n_act=4, n_virt=2, n_elec=2, Lc=5, Lx=0, ham="DC", seed=5),
    dict(n_core=2, n_act=6, n_virt=2, n_elec=3, Lc=3, Lx=2, ham="DCG", x_scale=0.05, seed=6),
    dict(n_core=2, n_act=8, n_virt=2, n_elec=4, Lc=3, das_size=[4, 4], das_min=[1, 1], das_max=[3, 3], seed=4),
    dict(n_core=2, n_act=6, n_virt=2, n_elec=3, Lc=3, das_size=[2, 2, 2], das_min=[1, 0, 0], das_max=[2, 2, 1],
         seed=7),
])
def test_e2_matches_fock_space_brute_force(case):
    """E0, E2 per root and class, and |Q| per class against H built from
    Jordan-Wigner operators (Eq. pt2 with Q from Sec. 2.3)."""
    p = tiny_problem(**case)
    o, c, _ = _ground(p)
    E0 = o.e0()
    _, ec, nc = o.e2(E0)
    E0b, eb, cb, _ = brute_e2(p, c)
    np.testing.assert_allclose(E0, E0b, rtol=0, atol=1e-11)
    np.testing.assert_allclose(ec, eb, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(nc, cb)


def test_e2_frozen_and_level_shift_match_brute_force():
    """Frozen core / virtual spinors (Sec. 2.5) and the real part of the
    imaginary level shift (Sec. 2.6) against the Fock-space sum."""
    p = tiny_problem(4, 4, 4, 2, Lc=4, Lx=2, ham="DCG", x_scale=0.05, n_frozen_core=2, n_frozen_virt=2,
                     level_shift_b=0.05, seed=8)
    o, c, _ = _ground(p)
    E0 = o.e0()
    _, ec, nc = o.e2(E0)
    _, eb, cb, _ = brute_e2(p, c, b=0.05)
    np.testing.assert_allclose(ec, eb, rtol=0, atol=1e-13)
    np.testing.assert_array_equal(nc, cb)


def test_matrix_elements_match_fock_space_and_are_hermitian():
    p = tiny_problem(2, 4, 4, 3, Lc=4, Lx=2, ham="DCB", x_scale=0.05, seed=9)
    o = Oracle(p)
    H = fock_hamiltonian(p).toarray()
    rng = np.random.default_rng(0)
    dets = [list(s) for s in combinations(range(p.n), 5)]
    for _ in range(400):
        K = dets[rng.integers(len(dets))]
        L = dets[rng.integers(len(dets))]
        if rng.random() < 0.5:       # bias towards connected pairs
            L = list(K)
            out = rng.choice(L)
            new = rng.choice([q for q in range(p.n) if q not in L])
            L = sorted([q for q in L if q != out] + [new])
        ki = sum(1 << q for q in K)
        li = sum(1 << q for q in L)
        v = o.hmat(K, L)
        assert abs(v - H[ki, li]) < 1e-13
        assert abs(v - np.conj(o.hmat(L, K))) < 1e-13


# ---------------------------------------------------------------- paper numbers

def _table3():
    rows = {}
    for line in open(os.path.join(GOLDEN, "table3_ndets.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        rows[f[0]] = f[1:]
    return rows


@pytest.mark.parametrize("system", ["Ne", "Ar", "Kr", "Xe"])
def test_external_space_size_matches_table3(system):
    """|Q| for all-electron (6e,8o) references over all positive-energy
    spinors reproduces the paper's nDets to its two printed figures."""
    spinors, electrons, na_e, na_s, ndets = _table3()[system]
    spinors, electrons, na_e, na_s = int(spinors), int(electrons), int(na_e), int(na_s)
    n_core = electrons - na_e
    p = tiny_problem(n_core, na_s, spinors - n_core - na_s, na_e, Lc=1)
    q = Oracle(p, use_eri_cache=False).count_q().sum()
    assert float(f"{q:.1e}") == float(ndets)


def test_reference_space_size_hbr():
    ne, ns, npd = _table3()["HBr_P"]
    p = tiny_problem(2, int(ns), 2, int(ne), Lc=1)
    assert Oracle(p).n_p == int(npd)


def test_pattern_count_equals_explicit_enumeration_das():
    p = tiny_problem(4, 12, 6, 6, Lc=2, das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2], seed=10)
    o, _, _ = _ground(p)
    _, _, nc = o.e2()
    np.testing.assert_array_equal(nc, o.count_q().astype(np.int64))


# ---------------------------------------------------------------- closed form

@pytest.mark.parametrize("full", [True, False])
def test_single_determinant_reduces_to_textbook_en_pt2(full):
    """Active space holding one determinant (N = n_act or N = 0): E2 is the
    single-reference Epstein-Nesbet sum over singles and doubles."""
    nc, na, nv = 4, 4, 6
    p = tiny_problem(nc, na, nv, na if full else 0, Lc=5, Lx=3, ham="DCB", x_scale=0.05, seed=11,
                     n_frozen_core=2)
    o, c, _ = _ground(p, 1)
    E2 = o.e2()[0][0]
    _, g = integrals(p)
    n = p.n
    occ = list(range(nc + (na if full else 0)))
    vir = [q for q in range(n) if q not in occ]
    corr_occ = [i for i in occ if not p.frozen[i]]
    G = np.real(np.einsum("pqpq->pq", g))
    eh = np.array([p.h[q, q].real + sum(G[q, k] for k in occ) for q in range(n)])
    ref = 0.0
    for i in corr_occ:
        for a in vir:
            f = p.h[a, i] + sum(g[a, k, i, k] for k in occ)
            ref += abs(f) ** 2 / (eh[i] - eh[a] + G[a, i])
    for i, j in combinations(corr_occ, 2):
        for a, b in combinations(vir, 2):
            D = eh[i] + eh[j] - eh[a] - eh[b] - G[i, j] - G[a, b] + G[a, i] + G[a, j] + G[b, i] + G[b, j]
            ref += abs(g[a, b, i, j]) ** 2 / D
    assert abs(E2 - ref) < 1e-12


# ---------------------------------------------------------------- symmetries

def test_integral_permutational_symmetry_and_hermiticity():
    p = tiny_problem(2, 4, 6, 2, Lc=5, Lx=4, ham="DCB", x_scale=0.1, seed=12)
    o = Oracle(p, use_eri_cache=False)
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b, c, d = rng.integers(0, p.n, 4)
        v = o.eri(a, b, c, d)
        scale = max(1.0, abs(v))
        assert abs(v - o.eri(c, d, a, b)) <= 1e-15 * scale
        assert abs(v - np.conj(o.eri(b, a, d, c))) <= 1e-15 * scale
        assert abs(v - np.conj(o.eri(d, c, b, a))) <= 1e-15 * scale
    assert np.abs(p.h - p.h.conj().T).max() == 0
    B, _ = p.factors()
    assert np.abs(B - B.conj().transpose(0, 2, 1)).max() == 0


def _time_reverse(prob, c):
    """T Psi for a CAS reference: T a+_(2k) T^-1 = a+_(2k+1),
    T a+_(2k+1) T^-1 = -a+_(2k), antiunitary."""
    na = prob.n_act
    out = np.zeros_like(c)
    for A in combinations(range(na), prob.n_elec):
        bits = sum(1 << t for t in A)
        tb, sign = 0, 1
        for t in A:
            tb |= 1 << (t ^ 1)
            if t & 1:
                sign = -sign
        full_pairs = sum(1 for k in range(0, na, 2) if (bits >> k) & 3 == 3)
        sign *= (-1) ** full_pairs
        out[:, p_address(prob, tb)] = sign * np.conj(c[:, p_address(prob, bits)])
    return out


@pytest.mark.parametrize("ham", ["DC", "DCG", "DCB"])
def test_time_reversal_invariance(ham):
    """Kramers-symmetric inputs (Gaunt/Breit factors time-reversal odd):
    E2(T Psi) = E2(Psi) for the reference and for an arbitrary vector."""
    p = tiny_problem(4, 6, 6, 3, Lc=4, Lx=3, ham=ham, x_scale=0.05, seed=13, time_reversal=True, n_roots=2,
                     n_frozen_core=2, n_frozen_virt=2)
    o, c, w = _ground(p)
    assert abs(w[1] - w[0]) < 1e-10        # odd electron count: Kramers pair
    rng = np.random.default_rng(2)
    for vec in (c, rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)):
        o.set_c(vec)
        e_a, ec_a, _ = o.e2()
        o.set_c(_time_reverse(p, vec))
        e_b, ec_b, _ = o.e2()
        np.testing.assert_allclose(ec_a, ec_b, rtol=0, atol=1e-12)


def test_spinor_phase_gauge_invariance():
    """p -> exp(i phi_p) p with c re-phased, and c -> exp(i theta) c, leave E2
    unchanged."""
    p = tiny_problem(2, 6, 6, 3, Lc=4, Lx=2, ham="DCG", x_scale=0.05, seed=14)
    o, c, _ = _ground(p, 1)
    e_ref = o.e2()[1]
    rng = np.random.default_rng(3)
    phi = rng.uniform(0, 2 * np.pi, p.n)
    U = np.exp(1j * phi)
    p2 = tiny_problem(2, 6, 6, 3, Lc=4, Lx=2, ham="DCG", x_scale=0.05, seed=14)
    p2.h = np.conj(U)[:, None] * p.h * U[None, :]
    p2.Bc = np.conj(U)[None, :, None] * p.Bc * U[None, None, :]
    p2.Bx = np.conj(U)[None, :, None] * p.Bx * U[None, None, :]
    c2 = c.copy()
    for A in combinations(range(p.n_act), p.n_elec):
        bits = sum(1 << t for t in A)
        ad = p_address(p, bits)
        c2[:, ad] *= np.exp(-1j * sum(phi[p.n_core + t] for t in A))
    o2 = Oracle(p2)
    o2.set_c(c2 * np.exp(0.7j))
    np.testing.assert_allclose(o2.e2()[1], e_ref, rtol=0, atol=1e-13)


def test_level_shift_limit():
    p = tiny_problem(2, 6, 8, 3, Lc=4, seed=15)
    o, c, _ = _ground(p, 1)
    E0 = o.e0()
    e0 = o.e2(E0)[0][0]
    o_small = Oracle(p, level_shift_b=1e-7)
    o_small.set_c(c)
    assert abs(o_small.e2(E0)[0][0] - e0) < 1e-12
    o_big = Oracle(p, level_shift_b=0.05)
    o_big.set_c(c)
    e_big = o_big.e2(E0)[0][0]
    assert e0 < e_big < 0                    # every denominator negative: shift damps each term


def test_frozen_spinors_give_partial_sums_and_raise_e2():
    """E2 with frozen spinors = the sum of the full-space terms whose
    determinants touch no frozen spinor (Sec. 2.5); all denominators are
    negative, so freezing never lowers E2."""
    kw = dict(Lc=4, Lx=2, ham="DCB", x_scale=0.05, seed=16)
    full = tiny_problem(4, 4, 6, 2, **kw)
    frz = tiny_problem(4, 4, 6, 2, n_frozen_core=2, n_frozen_virt=2, **kw)
    of, c, _ = _ground(full, 1)
    E0 = of.e0()
    ofz = Oracle(frz)
    ofz.set_c(c)
    _, ec_frz, nc_frz = ofz.e2(E0)
    # explicit list of the masked Q, evaluated on the full problem
    nh, hs, npp, ps, acts, cls = [], [], [], [], [], []
    corr_core = [k for k in range(4) if not frz.frozen[k]]
    corr_virt = [v for v in range(8, 14) if not frz.frozen[v]]
    for h in range(3):
        for pp in range(3):
            ne = 2 + h - pp
            if ne < 0 or ne > 4 or (h == 0 and pp == 0):
                continue
            for I in combinations(corr_core, h):
                for S in combinations(corr_virt, pp):
                    for A in combinations(range(4), ne):
                        nh.append(h); npp.append(pp)
                        hs.append(list(I) + [0] * (2 - h)); ps.append(list(S) + [0] * (2 - pp))
                        acts.append(sum(1 << t for t in A)); cls.append(3 * h + pp)
    V, D = of.couplings(E0, nh, hs, npp, ps, acts)
    terms = (np.abs(V[:, 0]) ** 2 / D[:, 0])
    part = np.bincount(cls, weights=terms, minlength=9)
    np.testing.assert_allclose(ec_frz[0], part, rtol=0, atol=1e-13)
    assert (D < 0).all()
    assert ofz.e2(E0)[0][0] > of.e2(E0)[0][0]


def test_reference_energy_is_lowest_eigenvalue():
    p = tiny_problem(2, 8, 4, 4, Lc=4, Lx=2, ham="DCG", x_scale=0.05, seed=17, n_roots=2)
    o, c, w = _ground(p)
    np.testing.assert_allclose(o.e0(), w, rtol=0, atol=1e-10)
    H = o.hpp()
    for m in range(2):
        assert np.linalg.norm(H @ c[m] - w[m] * c[m]) < 1e-10


def test_e2_is_invariant_to_the_scale_of_c():
    """Sec. 2.3 normalises the reference states; an unnormalised c gives the
    E2 of c/|c|."""
    p = tiny_problem(2, 6, 6, 3, Lc=4, seed=18)
    o, c, _ = _ground(p, 1)
    e_ref = o.e2()[1]
    o.set_c(3.7 * c)
    np.testing.assert_allclose(o.e2()[1], e_ref, rtol=1e-12, atol=1e-18)


# ---------------------------------------------------------------- gradient

def _fd4(f, d):
    return (-f(2 * d) + 8 * f(d) - 8 * f(-d) + f(-2 * d)) / (12 * d)


def _herm(rng, n):
    x = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (x + x.conj().T) / 2


@pytest.mark.parametrize("b", [0.0, 0.05])
def test_gradient_matches_central_differences(b):
    """dE2 along random Hermitian directions of h and of a Coulomb and a Breit
    factor, a complex direction of c (unnormalised, two roots with seeds),
    and the Breit multiplier lambda: 4th-order central differences, relative
    error <= 1e-7.  <c_m|cbar_m> = 0 (E2 is invariant to the scale and phase of c)."""
    import copy
    p = tiny_problem(4, 6, 6, 3, Lc=4, Lx=3, ham="DCB", x_scale=0.05, n_roots=2, seed=41, n_frozen_core=2,
                     level_shift_b=b)
    o, c, _ = _ground(p, 2)
    c = c * np.array([[1.3], [0.8j]])
    o.set_c(c)
    seed = np.array([1.0, 0.7])
    gh, gB, gw, gc = o.grad(seed=seed)
    rng = np.random.default_rng(5)

    def e2(q, cc):
        oo = Oracle(q)
        oo.set_c(cc)
        return seed @ oo.e2()[0]

    def check(fd, an):
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-3), (fd, an)

    dh = _herm(rng, p.n)
    def fh(t):
        q = copy.deepcopy(p)
        q.h = p.h + t * dh
        return e2(q, c)
    check(_fd4(fh, 1e-4), np.real(np.vdot(gh, dh)))
    for which, idx in (("c", 1), ("x", p.Bc.shape[0])):
        dB = _herm(rng, p.n)
        def fB(t):
            q = copy.deepcopy(p)
            if which == "c":
                q.Bc = p.Bc.copy()
                q.Bc[1] = p.Bc[1] + t * dB
            else:
                q.Bx = p.Bx.copy()
                q.Bx[0] = p.Bx[0] + t * dB
            return e2(q, c)
        check(_fd4(fB, 1e-4), np.real(np.vdot(gB[idx], dB)))
    dc = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    check(_fd4(lambda t: e2(p, c + t * dc), 1e-4), np.real(np.vdot(gc, dc)))
    for m in range(2):
        assert abs(np.vdot(c[m], gc[m])) < 1e-13
    def fl(t):
        q = copy.deepcopy(p)
        q.lam = p.lam + t
        return e2(q, c)
    check(_fd4(fl, 1e-3), np.dot(p.wx, gw[p.Bc.shape[0]:]))
