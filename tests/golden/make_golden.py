"""Write the oracle regression fixtures in this directory.

The paper prints no worked numerical example for the Wilson/clover operator
or the solver, so no fixture here is a paper value.  These files are written
by this script from the FP64 oracle alone (oracle/ and the seeded inputs of
synth/), and tests/test_golden.py checks that the oracle still reproduces
them: they guard the oracle against unintended change between commits.

    python tests/golden/make_golden.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import dirac, evenodd, solvers  # noqa: E402
from oracle.lattice import Lattice  # noqa: E402

DIMS = (2, 2, 2, 4)
KAPPA, CSW, EPS, SEED = 0.13, 1.0, 0.4, 2024


def cases():
    lat = Lattice(DIMS)
    U = synth.gauge_field(DIMS, EPS, SEED)
    psi = synth.gaussian_spinor(DIMS, SEED)
    eo = evenodd.EvenOdd(U, lat, KAPPA, CSW)
    x, info = solvers.bicgstab(lambda v: dirac.dirac(U, v, lat, KAPPA, CSW), psi, tol=1e-14)
    return {
        "wilson_D": dirac.wilson(U, psi, lat, KAPPA),
        "clover_D": dirac.dirac(U, psi, lat, KAPPA, CSW),
        "schur_Dhat": eo.schur(psi[lat.even]),
        "solution": x,
    }


def write():
    for name, arr in cases().items():
        flat = np.asarray(arr).reshape(-1)
        with open(os.path.join(HERE, f"{name}_2x2x2x4.txt"), "w") as f:
            f.write(f"# oracle {name}: lattice {DIMS}, kappa {KAPPA}, c_sw {CSW}, links exp({EPS} i A) seed {SEED},\n")
            f.write("# Gaussian source seed 2024 (synth); written by tests/golden/make_golden.py from oracle/ only.\n")
            f.write("# one complex number per line: real imag (canonical order [site][spin][colour])\n")
            for z in flat:
                f.write(f"{z.real:.17e} {z.imag:.17e}\n")


if __name__ == "__main__":
    write()
