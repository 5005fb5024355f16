"""Device status word (e2_query_status): conditions only the device sees.

* A NaN or an infinity in an input makes the energies non-finite in both
  arithmetics (FP64 and the emulated sliced form, whose slicers would otherwise
  turn a non-finite operand into finite digits) and sets the non-finite flag.
* An intruder state (Sec. 2.6): a one-body diagonal shifted on the host so that
  one external determinant's denominator E0 - H_KK vanishes; with b = 0 the
  intruder flag is set and min |D| of its class is below 1e-12 Eh; with the
  imaginary level shift b > 0 the same inputs give a finite energy and no flag.
* Clean inputs: no flag, and min |D| per class equals the smallest |D| the
  oracle finds over the class's external determinants (sampled exhaustively on
  a small case).

Every bad value is made on the host; the kernels only read it.
"""
import numpy as np
import pytest

from e2_inputs.synth import tiny_problem
from oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E2_OK, E2_ERR_NONFINITE, E2_ERR_INTRUDER = 0, 6, 7
NONFINITE, INTRUDER = 1, 2


def _plan(prob, c, sliced=False):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    plan = e2.E2Problem.from_problem(prob, n_roots=c.shape[0])
    plan.set_arithmetic(sliced)
    return e2, plan


def _problem(**kw):
    return tiny_problem(4, 8, 12, 4, Lc=5, Lx=3, ham="DCB", x_scale=0.05, seed=41, **kw)


def test_clean_inputs_raise_no_flag_and_min_D_matches_the_oracle():
    prob = _problem()
    o = Oracle(prob)
    c, _ = o.ground_state(1)
    E0 = o.e0()
    e2, plan = _plan(prob, c)
    t = e2.device_inputs(prob, c)
    plan.forward(**t)
    code, flags, mind = plan.status()
    assert code == E2_OK and flags == 0
    # oracle: the smallest |E0 - H_KK| over every external determinant of each class
    from itertools import combinations
    nc = list(range(prob.n_core))
    nv = list(range(prob.n_core + prob.n_act, prob.n))
    for h in range(3):
        for p in range(3):
            cls = 3 * h + p
            ne = prob.n_elec + h - p
            if cls == 0 or ne < 0 or ne > prob.n_act:
                assert not np.isfinite(mind[0, cls]) or plan.q_per_class[cls] == 0
                continue
            Ks = [(I, S, A) for I in combinations(nc, h) for S in combinations(nv, p)
                  for A in combinations(range(prob.n_act), ne)]
            nh = [h] * len(Ks)
            npp = [p] * len(Ks)
            hs = [list(I) + [0] * (2 - h) for I, _, _ in Ks]
            ps = [list(S) + [0] * (2 - p) for _, S, _ in Ks]
            acts = [sum(1 << a for a in A) for _, _, A in Ks]
            V, D = o.couplings(E0, nh, hs, npp, ps, acts)
            # class (2,2) counts the couplings with a non-zero <ab||ij>: all of them with these dense factors
            ref = float(np.abs(D[:, 0]).min())
            assert abs(mind[0, cls] - ref) <= 1e-10, (cls, mind[0, cls], ref)


@pytest.mark.parametrize("sliced", [False, True])
@pytest.mark.parametrize("where", ["B_c", "h_inf", "c"])
def test_non_finite_input_gives_non_finite_energy_and_flag(where, sliced):
    prob = _problem()
    c, _ = Oracle(prob).ground_state(1)
    e2, plan = _plan(prob, c, sliced=sliced)
    t = e2.device_inputs(prob, c)
    E2, _, _ = plan.forward(**t)
    torch.cuda.synchronize()
    assert np.isfinite(E2.cpu().numpy()).all()
    assert plan.status()[0] == E2_OK
    p, q = prob.n_core + 1, prob.n_core + prob.n_act + 3     # an active-virtual element
    if where == "B_c":
        t["B_c"][0, p, q] = complex(np.nan, 0.0)
        t["B_c"][0, q, p] = complex(np.nan, 0.0)
    elif where == "h_inf":
        t["h"][p, q] = complex(np.inf, 0.0)
        t["h"][q, p] = complex(np.inf, 0.0)
    else:
        t["c"][0, 3] = complex(np.nan, np.nan)
    E2, E2c, _ = plan.forward(**t)
    code, flags, _ = plan.status()
    assert not np.isfinite(E2.cpu().numpy()).all()
    assert flags & NONFINITE and code == E2_ERR_NONFINITE


def _intruder_inputs():
    """A problem and reference state whose class-(0,1) determinant K0 has
    E0 - H_KK = 0 up to rounding: the diagonal h_aa of K0's particle is raised
    by the oracle's D_K0 (every other determinant holding a moves with it)."""
    # small spinor energies keep the rounding of E0 - H_KK near 1e-14 Eh on both sides
    prob = _problem(core_ends=(-2.0, -1.5), virt_ends=(0.1, 5.0))
    o = Oracle(prob)
    c, _ = o.ground_state(1)
    E0 = o.e0()
    a = prob.n_core + prob.n_act + 4
    act = 0b1011      # 3 active electrons: class (0,1) has N - 1 = 3
    V, D = o.couplings(E0, [0], [[0, 0]], [1], [[a, 0]], [act])
    assert abs(V[0, 0]) > 1e-6
    prob.h = prob.h.copy()
    prob.h[a, a] += D[0, 0]
    o2 = Oracle(prob)
    o2.set_c(c)
    E0b = o2.e0()
    _, D2 = o2.couplings(E0b, [0], [[0, 0]], [1], [[a, 0]], [act])
    assert abs(D2[0, 0]) < 1e-12
    return prob, c


def test_intruder_denominator_sets_the_flag_and_the_level_shift_clears_it():
    prob, c = _intruder_inputs()
    e2, plan = _plan(prob, c)
    t = e2.device_inputs(prob, c)
    plan.forward(**t)
    code, flags, mind = plan.status()
    assert flags & INTRUDER
    assert code in (E2_ERR_INTRUDER, E2_ERR_NONFINITE)
    assert mind[0, 1] < 1e-12                  # class (0,1)
    # the imaginary level shift of Sec. 2.6 regularises the same inputs
    prob.level_shift_b = 0.05
    e2, plan_b = _plan(prob, c)
    E2, _, _ = plan_b.forward(**t)
    code, flags, mind = plan_b.status()
    assert code == E2_OK and flags == 0
    assert np.isfinite(E2.cpu().numpy()).all()
    assert mind[0, 1] < 1e-12                  # the diagnostic still reports the small denominator


def test_status_is_cleared_by_the_next_call():
    prob = _problem()
    c, _ = Oracle(prob).ground_state(1)
    e2, plan = _plan(prob, c)
    t = e2.device_inputs(prob, c)
    bad = dict(t)
    bad["h"] = t["h"].clone()
    bad["h"][0, 0] = complex(np.nan, 0.0)
    plan.forward(**bad)
    assert plan.status()[0] == E2_ERR_NONFINITE
    plan.forward(**t)
    assert plan.status()[:2] == (E2_OK, 0)


def _bins(D):
    """The documented decade bins of |D| (numpy, from the values the oracle gives)."""
    a = np.abs(D)
    k = np.full(a.shape, 17)
    k[a < 1e-12] = 0
    for q in range(1, 17):
        k[(a >= 10.0 ** (q - 13)) & (a < 10.0 ** (q - 12))] = q
    return k


def test_denominator_histogram_matches_the_oracle():
    """Every external determinant's |E0 - H_KK| counted once per class and
    decade; against the oracle's D of every determinant (a value within
    1e-9 relative of a decade edge may fall on either side)."""
    from itertools import combinations
    prob = _problem()
    o = Oracle(prob)
    c, _ = o.ground_state(1)
    E0 = o.e0()
    e2, plan = _plan(prob, c)
    t = e2.device_inputs(prob, c)
    hist = plan.denominator_histogram(**t).cpu().numpy()
    nc = list(range(prob.n_core))
    nv = list(range(prob.n_core + prob.n_act, prob.n))
    for cls in range(9):
        h, p = divmod(cls, 3)
        ne = prob.n_elec + h - p
        if cls == 0 or ne < 0 or ne > prob.n_act:
            assert hist[cls].sum() == 0
            continue
        Ks = [(I, S, A) for I in combinations(nc, h) for S in combinations(nv, p)
              for A in combinations(range(prob.n_act), ne)]
        _, D = o.couplings(E0, [h] * len(Ks), [list(I) + [0] * (2 - h) for I, _, _ in Ks], [p] * len(Ks),
                           [list(S) + [0] * (2 - p) for _, S, _ in Ks], [sum(1 << a for a in A) for _, _, A in Ks])
        ref = np.bincount(_bins(D[:, 0]), minlength=18)
        assert hist[cls].sum() == len(Ks) == plan.q_per_class[cls]
        edges = 10.0 ** np.arange(-12, 5)
        near = int(sum((np.abs(np.abs(D[:, 0]) - e) <= 1e-9 * e).sum() for e in edges))
        assert np.abs(hist[cls] - ref).sum() <= 2 * near, (cls, hist[cls], ref)


def test_denominator_histogram_flags_the_intruder():
    prob, c = _intruder_inputs()
    e2, plan = _plan(prob, c)
    t = e2.device_inputs(prob, c)
    hist = plan.denominator_histogram(**t).cpu().numpy()
    assert hist[1, 0] >= 1                     # class (0,1): the crafted |D| < 1e-12
    assert hist[[2, 4, 5, 6, 7, 8], 0].sum() == 0
