"""Per-coupling parity: V_K = <K|H|Psi> and D_K = E0 - H_KK of single external
determinants, written by the class kernels themselves (e2_probe_couplings:
one 64 x 64 tile of a dense class, a whole gather class), against the oracle's
explicit Q H P row and diagonal rule for the same determinants.

E2 needs only |V_K|^2, and the class factorisation may carry V_K with either
sign of the determinant convention, so the check is min(|V_gpu - V|,
|V_gpu + V|) per coupling (this still catches any error of magnitude or
complex phase, e.g. a conjugation or a sign inside the sum over the active
indices), and |D_gpu - D| <= 1e-10 Eh (the E0 bar).  Row and string orders
are the documented ones (rows_ref, strings_ref); a column-tiled class maps its
tile columns through the plan's column map.

Cases: the small CAS / DAS / frozen / two-root shapes, sampled tiles of the
full-size Ne-shaped DCG and Ar-shaped DCB DAS workloads (the benchmark's
launch configuration), and the Kr/Xe-shaped active space CAS(8e,24) with a
reduced core and virtual space, the last three with a seeded reference
vector concentrated on the P determinant of address 0 (no eigen-solve on
either side)."""
import numpy as np
import pytest

from e2_inputs import make_problem
from e2_inputs.synth import tiny_problem
from oracle import Oracle
from rows_ref import CLASSES, _row
from strings_ref import ClassStrings

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_D = 1e-10


def _plan(prob, n_roots):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    return e2, e2.E2Problem.from_problem(prob, n_roots=n_roots)


def _check(o, E0, prob, plan, cls, V, D, rows, ranks, lists, vscale):
    """Oracle V, D of every (row, string) of the block against the probe's."""
    cc = [k for k in range(prob.n_core) if not prob.frozen[k]]
    vc = [v for v in range(prob.n_core + prob.n_act, prob.n) if not prob.frozen[v]]
    strings = [lists[cls](r) for r in ranks]
    nh, hs, npp, ps, acts, where = [], [], [], [], [], []
    for i, row in enumerate(rows):
        H, Pp = _row(cls, row, cc, vc)
        for j, s in enumerate(strings):
            nh.append(len(H)), npp.append(len(Pp))
            hs.append(H + [0] * (2 - len(H))), ps.append(Pp + [0] * (2 - len(Pp)))
            acts.append(s)
            where.append((i, j))
    if not where:
        return 0
    Vo, Do = o.couplings(E0, nh, hs, npp, ps, acts)
    ii = np.array([w[0] for w in where])
    jj = np.array([w[1] for w in where])
    vg, dg = V[ii, jj], D[ii, jj]
    err = np.minimum(np.abs(vg - Vo[:, 0]), np.abs(vg + Vo[:, 0]))
    assert (err <= 1e-12 * vscale + 1e-10 * np.abs(Vo[:, 0])).all(), (cls, float(err.max()))
    assert (np.abs(dg - Do[:, 0]) <= TOL_D).all(), (cls, float(np.abs(dg - Do[:, 0]).max()))
    return len(where)


def _run(prob, c, tiles_per_class, seed=3):
    e2, plan = _plan(prob, c.shape[0])
    o = Oracle(prob, use_eri_cache=prob.n <= 96)
    o.set_c(c)
    E0 = o.e0()
    t = e2.device_inputs(prob, c)
    lists = {cls: ClassStrings(prob, *CLASSES[cls]) for cls in CLASSES}
    rng = np.random.default_rng(seed)
    vscale = 0.0
    checked = 0
    for cls in (2, 5, 7, 4, 6, 1, 3, 0):
        if plan.q_per_class[cls] == 0:
            continue
        nA = lists[cls].n
        if cls in (1, 3, 0):                              # gather class: the whole class
            V, D = plan.probe_couplings(cls, **t)
            V, D = V.cpu().numpy(), D.cpu().numpy()
            vscale = max(vscale, float(np.abs(V).max()))
            rows = list(range(V.shape[0]))
            ranks = list(range(nA))
            if V.shape[0] * nA > 4096:                    # a seeded sample of rows and strings
                rows = sorted({0, V.shape[0] - 1} | set(rng.integers(V.shape[0], size=4).tolist()))
                ranks = sorted({0, nA - 1} | set(rng.integers(nA, size=256).tolist()))
                V, D = V[np.ix_(rows, ranks)], D[np.ix_(rows, ranks)]
            checked += _check(o, E0, prob, plan, cls, V, D, rows, ranks, lists, vscale)
            continue
        M = int(round(plan.q_per_class[cls] / nA))
        rt = (M + 63) // 64
        tiles, _, used = plan.class_tiles(cls)
        perm = plan.class_tiles_plan(cls)[0] if used else None
        ct = tiles if used else (nA + 63) // 64
        picks = {(rt - 1, ct - 1), (0, 0)}
        picks |= {(int(rng.integers(rt)), int(rng.integers(ct))) for _ in range(tiles_per_class - 2)}
        for tm, tn in sorted(picks):
            V, D = plan.probe_couplings(cls, **t, tile_m=tm, tile_n=tn)
            V, D = V.cpu().numpy(), D.cpu().numpy()
            vscale = max(vscale, float(np.abs(V).max()))
            rows = list(range(64 * tm, min(64 * tm + 64, M)))
            if perm is None:
                cols = [(j, 64 * tn + j) for j in range(64) if 64 * tn + j < nA]
            else:
                cols = [(j, int(perm[64 * tn + j])) for j in range(64) if perm[64 * tn + j] >= 0]
            Vb = V[:len(rows)][:, [j for j, _ in cols]]
            Db = D[:len(rows)][:, [j for j, _ in cols]]
            checked += _check(o, E0, prob, plan, cls, Vb, Db, rows, [r for _, r in cols], lists, vscale)
    return checked


SMALL = {
    "dc_small": lambda: make_problem("dc_small"),
    "dcb_two_roots_frozen": lambda: tiny_problem(6, 8, 14, 4, Lc=6, Lx=4, ham="DCB", x_scale=0.05, n_roots=2,
                                                 n_frozen_core=2, n_frozen_virt=3, seed=21),
    "dcg_odd_electrons": lambda: tiny_problem(4, 10, 12, 5, Lc=5, Lx=3, ham="DCG", x_scale=0.05, seed=22),
    "das_three_subspaces": lambda: tiny_problem(4, 12, 10, 6, Lc=5, Lx=2, ham="DCB", x_scale=0.05,
                                                das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2], seed=23),
}


@pytest.mark.parametrize("name", list(SMALL))
def test_single_couplings_match_the_oracle(name):
    prob = SMALL[name]()
    o = Oracle(prob)
    c, _ = o.ground_state(prob.n_roots)
    assert _run(prob, c[:1], tiles_per_class=4) > 1000


def _concentrated_c(prob, seed):
    """A seeded reference vector: weight 1 on the P determinant of address 0
    (for a CAS the lowest active spinors filled), plus 0.05 complex N(0,1)
    everywhere, normalised.  Made from the seed alone, the same on both
    sides."""
    from e2_inputs.synth import n_p_space
    n_p = n_p_space(prob.das_size, prob.das_min, prob.das_max, prob.n_elec)
    rng = np.random.default_rng(seed)
    c = 0.05 * (rng.standard_normal((1, n_p)) + 1j * rng.standard_normal((1, n_p)))
    c[0, 0] += 1.0
    return c / np.linalg.norm(c)


@pytest.mark.parametrize("config", ["ne_dcg", "ar_dcb_das"])
def test_single_couplings_at_full_size(config):
    prob = make_problem(config)
    assert _run(prob, _concentrated_c(prob, 17), tiles_per_class=3) > 20000


def test_single_couplings_at_the_kr_xe_active_shape():
    """The Kr- and Xe-shaped active space CAS(8e,24) (735,471 reference
    determinants, 1.96 million strings in the (2,0) list) with a reduced core
    (4) and virtual (16) space and factor set (8 + 4): sampled tiles of every
    dense class and samples of the gather classes."""
    prob = tiny_problem(4, 24, 16, 8, Lc=8, Lx=4, ham="DCB", x_scale=4e-3, core_ends=(-1280.0, -2.5),
                        virt_ends=(0.1, 800.0), seed=68)
    assert _run(prob, _concentrated_c(prob, 19), tiles_per_class=3) > 20000
