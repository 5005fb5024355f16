"""The C ABI without a GPU: the library loads, exports every entry point that
include/e2.h declares, validates descriptors on the host, and plans the same
external-space sizes as the oracle counts."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from e2_inputs.synth import tiny_problem, make_problem
from oracle import Oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    e2build.build()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*(?:E2_API\s+)?(?:e2_status|const char\*)\s+(e2_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_library_exports_every_declared_entry_point():
    lib = C.CDLL(e2.LIB_PATH)
    names = _declared()
    assert "e2_forward" in names and "e2_problem_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    lib = e2.load()
    for s in range(10):
        assert lib.e2_status_string(s) and lib.e2_status_string(s) != b"unknown status"


@pytest.mark.parametrize("kw,err", [
    (dict(n_core=2, n_active=0, n_virt=2, n_elec=0), "inconsistent"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=5), "inconsistent"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, ham="DC", L_extra=3), "invalid"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, das_size=[2, 3], das_min=[0, 0], das_max=[2, 2]), "inconsistent"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, das_size=[2, 2], das_min=[2, 2], das_max=[2, 2]), "inconsistent"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, n_roots=0), "invalid"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, level_shift_b=-1.0), "invalid"),
    (dict(n_core=2, n_active=4, n_virt=2, n_elec=2, frozen=[0, 0, 1, 0, 0, 0, 0, 0]), "inconsistent"),
])
def test_descriptor_validation(kw, err):
    with pytest.raises(e2.E2Error, match=err):
        e2.E2Problem(**kw)


@pytest.mark.parametrize("case", [
    dict(n_core=4, n_act=12, n_virt=40, n_elec=6),
    dict(n_core=4, n_act=8, n_virt=10, n_elec=4, n_frozen_core=2, n_frozen_virt=3),
    dict(n_core=4, n_act=12, n_virt=6, n_elec=6, das_size=[4, 4, 4], das_min=[2, 0, 0], das_max=[4, 4, 2]),
    dict(n_core=2, n_act=6, n_virt=2, n_elec=3, das_size=[2, 2, 2], das_min=[1, 0, 0], das_max=[2, 2, 1]),
])
def test_plan_sizes_match_oracle_counts(case):
    p = tiny_problem(Lc=1, **case)
    plan = e2.E2Problem.from_problem(p)
    o = Oracle(p, use_eri_cache=False)
    assert plan.n_p == o.n_p
    np.testing.assert_array_equal(plan.q_per_class, o.count_q())


def test_plan_sizes_of_the_workload_shapes():
    """|Q| per root of the Ne- and Ar-shaped workloads (no arrays needed)."""
    for name, q in [("dc_small", 7557198), ("ne_dcg", 880539088)]:
        kw = dict(make_problem.__globals__["CONFIGS"][name])
        p = e2.E2Problem(kw["n_core"], kw["n_act"], kw["n_virt"], kw["n_elec"], ham=kw["ham"],
                         L_coulomb=kw["Lc"], L_extra=kw["Lx"] if kw["ham"] != "DC" else 0)
        assert int(p.q_per_class.sum()) == q
