"""The oracle: TEST INFRASTRUCTURE ONLY.

A plain, slow CPU evaluation of the Epstein–Nesbet second-order energy
(Sec. 2.3, Eq. pt2; Sec. 2.4, Eq. pt2en) that builds Q H P explicitly with
generic Slater–Condon rules over bitset determinants.  It shares no code with
the GPU library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.
"""
from .oracle import Oracle, build, lib_path

__all__ = ["Oracle", "build", "lib_path"]
