"""Tuning cache (e2_tuning_save / e2_tuning_load), host only: the column-tile
choices of a problem survive a save and a load into a fresh plan of the same
shape; a plan of another shape finds no entry and keeps its defaults; the
last matching entry wins; a missing file is reported, not an error."""
import os

import pytest

import paper_2608_11529_b300 as e2
from paper_2608_11529_b300 import build as e2build
from e2_inputs import make_problem


def _plan(**over):
    e2build.build()
    return e2.E2Problem.from_problem(make_problem("dc_small", **over))


def test_choices_round_trip(tmp_path):
    path = str(tmp_path / "tune.txt")
    a = _plan()
    tiled = [k for k in range(9) if a.class_tiles(k)[0]]
    assert tiled
    flip = {k: not a.class_tiles(k)[2] for k in tiled}
    for k, on in flip.items():
        a.set_class_tiles(k, on)
    a.tuning_save(path)
    b = _plan()
    assert all(b.class_tiles(k)[2] != flip[k] for k in tiled)      # fresh plan: the defaults
    assert b.tuning_load(path)
    assert all(b.class_tiles(k)[2] == flip[k] for k in tiled)
    # the last entry for a shape wins
    for k in tiled:
        a.set_class_tiles(k, not flip[k])
    a.tuning_save(path)
    c = _plan()
    assert c.tuning_load(path)
    assert all(c.class_tiles(k)[2] == (not flip[k]) for k in tiled)


def test_other_shapes_and_missing_files(tmp_path):
    path = str(tmp_path / "tune.txt")
    _plan().tuning_save(path)
    other = _plan(n_virt=42)
    assert not other.tuning_load(path)
    assert not other.tuning_load(str(tmp_path / "absent.txt"))
    assert e2.load().e2_tuning_save(other._h, os.fsencode(str(tmp_path / "no_dir" / "x.txt"))) == 1
