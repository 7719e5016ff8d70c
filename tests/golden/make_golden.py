"""Write the oracle regression fixtures in this directory.

The paper prints no worked numerical example for any of its operators or
solvers, so no fixture here is a paper value.  These files are written
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
from oracle import dirac, domainwall, evenodd, multigrid, solvers, staggered  # noqa: E402
from oracle.lattice import Lattice  # noqa: E402

DIMS = (2, 2, 2, 4)
KAPPA, CSW, EPS, SEED = 0.13, 1.0, 0.4, 2024


def cases():
    lat = Lattice(DIMS)
    U = synth.gauge_field(DIMS, EPS, SEED)
    psi = synth.gaussian_spinor(DIMS, SEED)
    eo = evenodd.EvenOdd(U, lat, KAPPA, CSW)
    x, info = solvers.bicgstab(lambda v: dirac.dirac(U, v, lat, KAPPA, CSW), psi, tol=1e-14)
    # Moebius (Ls = 4, M5 = 1.8, b = 1.5, c = 0.5, m_f = 0.1) and staggered (m = 0.1)
    # on the same field; their sources are slices of a seeded Gaussian spinor
    mob = domainwall.Mobius(U, lat, 4, 1.8, 1.5, 0.5, 0.1)
    psi5 = synth.gaussian_spinor(DIMS, SEED, nrhs=4)
    stg = staggered.Staggered(U, lat, 0.1)
    chi = psi[:, 0, :]
    # two-level multigrid: blocks 1x1x1x2 (2^4 coarse sites), the two null
    # vectors a seeded Gaussian pair; the cycle (exact coarse solve, 2 SAP
    # cycles of 4 MR steps) and the even-odd coarse solve of the restricted source
    mg = multigrid.Multigrid(U, lat, KAPPA, CSW, (1, 1, 1, 2), synth.gaussian_spinor(DIMS, SEED + 1, nrhs=2))
    mg_eo, _ = mg.coarse_evenodd_solve(mg.restrict(psi), tol=1e-14)
    return {
        "wilson_D": dirac.wilson(U, psi, lat, KAPPA),
        "clover_D": dirac.dirac(U, psi, lat, KAPPA, CSW),
        "schur_Dhat": eo.schur(psi[lat.even]),
        "solution": x,
        "mobius_D": mob.full(psi5),
        "mobius_Dhat_dag": mob.schur_dag(psi5[:, lat.even]),
        "staggered_D": stg.full(chi),
        "staggered_Dhat": stg.schur(chi[lat.even]),
        "mg_cycle": mg.cycle(psi, 2, 4),
        "mg_coarse_eo_solve": mg_eo,
    }


def write():
    for name, arr in cases().items():
        flat = np.asarray(arr).reshape(-1)
        with open(os.path.join(HERE, f"{name}_2x2x2x4.txt"), "w") as f:
            f.write(f"# oracle {name}: lattice {DIMS}, kappa {KAPPA}, c_sw {CSW}, links exp({EPS} i A) seed {SEED},\n")
            f.write("# Moebius Ls 4, M5 1.8, b 1.5, c 0.5, m_f 0.1; staggered m 0.1 (spin-0 components of the source);\n")
            f.write("# multigrid blocks 1x1x1x2, null vectors Gaussian seed 2025 (2 of them), 2 SAP cycles x 4 MR steps;\n")
            f.write("# Gaussian source seed 2024 (synth); written by tests/golden/make_golden.py from oracle/ only.\n")
            f.write("# one complex number per line: real imag (canonical order [site][spin][colour])\n")
            for z in flat:
                f.write(f"{z.real:.17e} {z.imag:.17e}\n")


if __name__ == "__main__":
    write()
