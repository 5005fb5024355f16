"""Host plan of the column tiles (no GPU): every class string lands in exactly
one tile, and every table row that is structurally non-zero for a string of a
tile is among that tile's compacted rows.  Without the second property the
compacted contraction would drop couplings.

The string order comes from the documented address convention (strings_ref).
The non-zero rules are stated here from the operator definitions:
  D^{tu}_A    = <A| a_u a_t |Psi>     needs t, u empty in A      (class (0,2))
  D^{t+u+}_A  = <A| a+_t a+_u |Psi>   needs t, u occupied in A   (class (2,0))
  D^t_A       = <A| a_t |Psi>         needs t empty in A         (class (1,2))
  D^{t+u}_A   = <A| a+_t a_u |Psi>    needs t occupied, u empty, or t = u
                occupied; row 0 is c_A itself                     (class (1,1))
"""
import numpy as np
import pytest

from strings_ref import ClassStrings

CLASS_HP = {2: (0, 2), 6: (2, 0), 5: (1, 2), 4: (1, 1)}
GRAN = {2: 8, 6: 8, 4: 8, 5: 4}


def _rows_nonzero(cls, na, A):
    """Boolean vector over the coupling-table rows of class cls for string A."""
    occ = np.array([(A >> t) & 1 for t in range(na)], bool)
    if cls in (2, 6):
        out = []
        for u in range(1, na):
            for t in range(u):
                out.append((not occ[t] and not occ[u]) if cls == 2 else (occ[t] and occ[u]))
        return np.array(out, bool)
    if cls == 5:
        return ~occ
    rows = [True]
    for t in range(na):
        for u in range(na):
            rows.append(bool(occ[t]) if t == u else bool(occ[t] and not occ[u]))
    return np.array(rows, bool)


def _shape(kind):
    from e2_inputs.synth import tiny_problem
    if kind == "cas":
        return tiny_problem(4, 12, 10, 6, Lc=2, seed=81)
    if kind == "das":
        return tiny_problem(4, 12, 10, 6, Lc=2, das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2], seed=82)
    if kind == "ne_active":   # the benchmark's CAS(8e,16) with a small external space
        return tiny_problem(2, 16, 6, 8, Lc=2, seed=83)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["cas", "das", "ne_active"])
def test_column_tiles_cover_every_structural_nonzero(kind):
    import paper_2608_11529_b300 as e2
    from paper_2608_11529_b300 import build as e2build
    e2build.build()
    prob = _shape(kind)
    plan = e2.E2Problem.from_problem(prob)
    na = prob.n_act
    checked = 0
    for cls, (h, p) in CLASS_HP.items():
        tiles, krows, _ = plan.class_tiles(cls)
        if tiles == 0:
            continue
        perm, tdesc, klist = plan.class_tiles_plan(cls)
        lst = ClassStrings(prob, h, p)
        valid = perm[perm >= 0]
        # a permutation of the class's strings, padding only after the last string
        assert sorted(valid.tolist()) == list(range(lst.n))
        assert (perm[:lst.n] >= 0).all() and (perm[lst.n:] < 0).all()
        assert tiles == (lst.n + 63) // 64
        koff = 0
        for j in range(tiles):
            k0, klen, ktrue, _ = tdesc[j]
            assert k0 == koff and klen % GRAN[cls] == 0 and 0 <= ktrue <= klen
            rows = klist[k0:k0 + ktrue]
            assert (np.diff(rows) > 0).all()
            assert (klist[k0 + ktrue:k0 + klen] == 0).all()
            need = np.zeros(len(_rows_nonzero(cls, na, 0)), bool)
            for s in perm[64 * j:64 * j + 64]:
                if s >= 0:
                    need |= _rows_nonzero(cls, na, lst(int(s)))
            assert set(np.nonzero(need)[0].tolist()) <= set(rows.tolist()), (cls, j)
            koff += klen
        assert koff == krows
        checked += 1
    assert checked >= 3
