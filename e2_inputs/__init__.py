"""Seeded synthetic inputs for the Epstein–Nesbet second-order energy.

This module is shared by the oracle (tests) and the GPU library (tests,
bench).  It draws numbers and lays them out; it holds none of the method's
arithmetic (no integrals, no matrix elements, no determinants).

Every array comes from ``numpy.random.default_rng([config_id, stream, ...])``
so each piece can be regenerated independently and lazily.

Spinor order (global index): [core | active | virtual]; within each block the
Kramers pairs sit at (2k, 2k+1).  Frozen core spinors are the lowest core
indices, frozen virtual spinors the highest virtual indices (Sec. 2.5 freezes
deep core and high-lying virtuals).
"""
from .synth import (Problem, CONFIGS, make_problem, tiny_problem, das_patterns,
                    n_p_space, pattern_count)

__all__ = ["Problem", "CONFIGS", "make_problem", "tiny_problem", "das_patterns",
           "n_p_space", "pattern_count"]
