"""Pin of the oracle's core / virtual DAS subspaces with hole / particle
limits (Sec. 2.4, Fig. 1): against the Jordan-Wigner brute force with the
same restriction of Q written here from its definition (count the holes of
each core block and the particles of each virtual block of the Fock state),
per root and class, E2 and |Q|; limits of 2 change nothing; and E2 with limits
is the full E2 minus exactly the excluded determinants' terms."""
import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from jw_fock import brute_e2
from oracle import Oracle

CORE, CORE_MAX = [2, 2], [1, 2]
VIRT, VIRT_MAX = [2, 4], [1, 2]


def _allowed(prob):
    nc, v0 = prob.n_core, prob.n_core + prob.n_act

    def ok(K):
        at = 0
        for size, lim in zip(CORE, CORE_MAX):
            holes = sum(1 for p in range(at, at + size) if not (K >> p) & 1)
            if holes > lim:
                return False
            at += size
        at = v0
        for size, lim in zip(VIRT, VIRT_MAX):
            parts = sum(1 for p in range(at, at + size) if (K >> p) & 1)
            if parts > lim:
                return False
            at += size
        return True
    assert sum(CORE) == nc and sum(VIRT) == prob.n_virt
    return ok


CASES = {
    "cas": lambda: tiny_problem(4, 4, 6, 2, Lc=3, seed=71),
    "dcb_two_roots": lambda: tiny_problem(4, 4, 6, 2, Lc=3, Lx=2, ham="DCB", x_scale=0.05, n_roots=2, seed=72),
    "level_shift": lambda: tiny_problem(4, 4, 6, 2, Lc=3, level_shift_b=0.1, seed=73),
}


@pytest.mark.parametrize("name", list(CASES))
def test_limits_match_the_brute_force(name):
    prob = CASES[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    o.set_external_das(CORE, CORE_MAX, VIRT, VIRT_MAX)
    E0 = o.e0()
    _, ec, nc = o.e2(E0)
    bE0, be2, bcount, _ = brute_e2(prob, c, b=prob.level_shift_b, allowed=_allowed(prob))
    np.testing.assert_allclose(E0, bE0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ec, be2, rtol=0, atol=1e-12)
    assert np.array_equal(nc, bcount)
    assert np.array_equal(o.count_q(), bcount.astype(float))
    assert bcount[8] < brute_e2(prob, c, b=prob.level_shift_b)[2][8]   # the limits remove (2,2) determinants


def test_limits_of_two_change_nothing_and_removed_terms_add_up():
    prob = CASES["cas"]()
    o = Oracle(prob)
    c, _ = o.ground_state(1)
    E0 = o.e0()
    _, full, nfull = o.e2(E0)
    o.set_external_das(CORE, [2, 2], VIRT, [2, 2])
    _, same, nsame = o.e2(E0)
    assert np.array_equal(same, full) and np.array_equal(nsame, nfull)
    o.set_external_das(CORE, CORE_MAX, VIRT, VIRT_MAX)
    _, lim, _ = o.e2(E0)
    # the excluded determinants' terms, summed explicitly
    from itertools import combinations
    ok = _allowed(prob)
    v0 = prob.n_core + prob.n_act
    excl = np.zeros(9)
    for h in range(3):
        for p in range(3):
            ne = prob.n_elec + h - p
            if (h, p) == (0, 0) or not 0 <= ne <= prob.n_act:
                continue
            Ks = []
            for I in combinations(range(prob.n_core), h):
                for S in combinations(range(v0, prob.n), p):
                    for A in combinations(range(prob.n_act), ne):
                        occ = ((1 << prob.n_core) - 1) & ~sum(1 << i for i in I)
                        occ |= sum(1 << (prob.n_core + t) for t in A) | sum(1 << s for s in S)
                        if not ok(occ):
                            Ks.append((I, S, A))
            if not Ks:
                continue
            V, D = o.couplings(E0, [h] * len(Ks), [list(I) + [0] * (2 - h) for I, _, _ in Ks], [p] * len(Ks),
                               [list(S) + [0] * (2 - p) for _, S, _ in Ks],
                               [sum(1 << t for t in A) for _, _, A in Ks])
            excl[3 * h + p] = float(np.sum(np.abs(V[:, 0]) ** 2 / D[:, 0]))
    np.testing.assert_allclose(lim[0], full[0] - excl, rtol=0, atol=1e-12)
