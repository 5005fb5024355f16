"""Write ar_dcb_das_reference.npz: the reference state of the Ar-shaped DCB
DAS workload (8 core + three active subspaces of 8 spinors holding 10
electrons, N_P = 40,608, 400 virtual spinors, 600 Coulomb + 300 Breit
factors) and its reference energy, both from the oracle alone.

The reference state is the lowest eigenvector of P H P (the CASCI / DAS-CI
reference of Sec. 2.2-2.3), its largest entry made real positive; the energy
is its Rayleigh quotient E0 = <Psi|H|Psi>/<Psi|Psi> (Sec. 2.3).  Building
P H P with the oracle's explicit Slater-Condon rows takes tens of minutes at
this size, which is why the full-size parity test reads the state from this
file instead of solving for it.  The file also records a digest of the
workload's inputs, so that a change of the input generator is caught.

    python tests/golden/make_ar_reference.py
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ar_dcb_das_reference.npz")


def inputs_digest(prob):
    """sha256 over the workload's inputs (h, factors, weights, start vectors)."""
    h = hashlib.sha256()
    for a in (prob.h, prob.Bc, prob.Bx, prob.wx, prob.X0):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def main():
    from e2_inputs import make_problem
    from oracle import Oracle
    t0 = time.time()
    prob = make_problem("ar_dcb_das")
    o = Oracle(prob, use_eri_cache=False)
    c, w = o.ground_state(1)
    E0 = o.e0()
    np.savez(OUT, c=c, E0=E0, eigenvalue=w, digest=np.array(inputs_digest(prob)))
    print(f"wrote {OUT}: E0 = {E0}, lowest eigenvalue = {w}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
