"""Pin of the oracle's coupling tensors D^x_A = <A|x|Psi> (Sec. 2.4, Eq.
sumsigma: the <K|E_pq|L> C_L factors restricted to the active space) against
a Jordan-Wigner Fock-space brute force that shares nothing with the oracle's
bitset code: |Psi> is placed in the 2^n Fock space, x is a product of
Jordan-Wigner matrices, and D^x_A is the amplitude of |A> (core full,
virtuals empty) in x|Psi>.  Every entry is exactly +-c_L or 0, so the
comparison is bit for bit.  Also checked: the diagonal sum rule
sum_A |D^t_A|^2 = <Psi|a+_t a_t|Psi> (the occupation of t) and that entries
vanish for operators that cannot reach P."""
from itertools import combinations

import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from jw_fock import annihilators, p_address
from oracle import Oracle

CASES = {
    "cas": lambda: tiny_problem(2, 8, 2, 4, Lc=2, seed=51),
    "cas_odd": lambda: tiny_problem(2, 8, 2, 3, Lc=2, seed=52),
    "das": lambda: tiny_problem(2, 12, 0, 4, Lc=2, das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2],
                                seed=53),
}
FAMILY_ELECTRONS = {"t": -1, "t+": 1, "tu": -2, "t+u+": 2, "t+u": 0}


def _rows(family, na):
    """(operator factors, row) in the oracle's row order; factors act right to left."""
    out = []
    if family == "t":
        out = [([("a", t)], t) for t in range(na)]
    elif family == "t+":
        out = [([("c", t)], t) for t in range(na)]
    elif family in ("tu", "t+u+"):
        for u in range(na):
            for t in range(u):
                r = u * (u - 1) // 2 + t
                # x = a_u a_t  (apply a_t first)  |  x = a+_t a+_u (apply a+_u first)
                out.append(([("a", t), ("a", u)] if family == "tu" else [("c", u), ("c", t)], r))
    else:
        out.append(([], 0))
        for t in range(na):
            for u in range(na):
                out.append(([("a", u), ("c", t)], 1 + t * na + u))
    return out


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("family", list(FAMILY_ELECTRONS))
def test_dtables_equal_jordan_wigner_amplitudes_bit_for_bit(name, family):
    prob = CASES[name]()
    n, nc, na = prob.n, prob.n_core, prob.n_act
    o = Oracle(prob)
    rng = np.random.default_rng(7)
    c = rng.standard_normal((1, o.n_p)) + 1j * rng.standard_normal((1, o.n_p))
    o.set_c(c)
    # |Psi> in the Fock space
    core = (1 << nc) - 1
    psi = np.zeros(1 << n, complex)
    for A in combinations(range(na), prob.n_elec):
        bits = sum(1 << t for t in A)
        ad = p_address(prob, bits)
        if ad >= 0:
            psi[core | (bits << nc)] = c[0, ad]
    a = annihilators(n)
    ne = prob.n_elec + FAMILY_ELECTRONS[family]
    strings = [sum(1 << t for t in A) for A in combinations(range(na), ne)] if 0 <= ne <= na else []
    if not strings:
        pytest.skip("no strings of this electron count")
    got = o.dtable(family, strings)
    for ops, r in _rows(family, na):
        v = psi.copy()
        for kind, t in ops:
            m = a[nc + t] if kind == "a" else a[nc + t].T.tocsr()
            v = m @ v
        ref = np.array([v[core | (A << nc)] for A in strings])
        assert np.array_equal(got[r], ref), (family, r)


@pytest.mark.parametrize("name", list(CASES))
def test_occupation_sum_rule(name):
    prob = CASES[name]()
    o = Oracle(prob)
    rng = np.random.default_rng(8)
    c = rng.standard_normal((1, o.n_p)) + 1j * rng.standard_normal((1, o.n_p))
    o.set_c(c)
    na, N = prob.n_act, prob.n_elec
    minus = [sum(1 << t for t in A) for A in combinations(range(na), N - 1)]
    same = [sum(1 << t for t in A) for A in combinations(range(na), N)]
    Dt = o.dtable("t", minus)
    Dn = o.dtable("t+u", same)
    for t in range(na):
        occ = np.sum(np.abs(Dt[t]) ** 2)
        # <Psi|a+_t a_t|Psi> = sum_A conj(c_A) <A|a+_t a_t|Psi>
        num = np.sum(np.conj(Dn[0]) * Dn[1 + t * na + t]).real
        assert occ == pytest.approx(num, rel=1e-13)
