"""B300 (sm_103a) Epstein-Nesbet second-order energy of a multiconfigurational
four-component reference (4C-MRPT2, Sec. 2.3-2.6).

The compute path is ``libe2.so`` (C ABI declared in ``include/e2.h``); this
package is its Python binding.
"""
from ._lib import E2Problem, E2Batch, E2Error, device_inputs, fp64_peak, load, CLASS_NAMES, NCLASS, LIB_PATH
from .autograd import E2Function, e2_energy

__all__ = ["E2Problem", "E2Batch", "E2Error", "device_inputs", "fp64_peak", "load", "CLASS_NAMES", "NCLASS", "LIB_PATH",
           "E2Function", "e2_energy"]
