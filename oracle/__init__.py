"""FP64 CPU oracle for the even-odd Wilson/clover and Moebius domain-wall solver paths.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
definition that the CUDA library is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference legs of
``bench.py`` may import it.  The product library never calls it and shares no
code with it.

Contents (each function cites the passage of the paper it follows; where the
paper is silent, the docstring states the reading taken):

* ``lattice``  -- site indexing, parity and neighbour maps with boundary phases;
* ``gamma``    -- the gamma matrices (chiral basis) and sigma_{mu nu};
* ``dirac``    -- hopping term H, Wilson D = 1 - kappa H, the clover term T,
                  full D = T - kappa H (Sec. 2 of the paper);
* ``evenodd``  -- the blocks D_ee, D_oo, D_eo, D_oe and the Schur operator
                  D^(eo) = 1 - D_ee^-1 D_eo D_oo^-1 D_oe (Eq. 1), source
                  preparation and odd-site reconstruction;
* ``domainwall`` -- the Moebius domain-wall operator (Sec. 2), its even-odd
                  blocks over four-dimensional parity with the fifth
                  coordinate as an inner index, the Schur operator and its
                  adjoint;
* ``staggered`` -- the staggered operator (Sec. 2) with its even-odd blocks
                  and the Hermitian positive definite even system solved by CG;
* ``multigrid`` -- the two-level multigrid of Sec. 3 (aggregation by blocks
                  and chirality, P^dag D P, SAP with minimal-residual block
                  solves, the cycle, Flexible BiCGStab);
* ``solvers``  -- BiCGStab (van der Vorst) as named in Sec. 3, CG and CG on
                  the normal equations (the domain-wall solver of Fig. 7),
                  dense matrices by their matrix elements and dense LU solves.

Arrays are complex128 in the canonical layouts of ``synth``: spinors
``(V, 4, 3)``, links ``(4, V, 3, 3)``, half-lattice vectors ``(V/2, 4, 3)``
ordered by lexicographic index among the sites of one parity.

Parity status: every function here is pinned by a CPU test against a closed
form, an invariant or a library routine (see tests/test_oracle_pins.py);
none is marked "parity unpinned" except the overall sign/normalisation of the
clover term, which is a convention the paper does not state (the abelian-flux
closed form pins the reading taken, not the paper).  The domain-wall operator
is pinned by the overlap relation (its boundary-field operator equals the
polar approximation of the sign function of the Moebius kernel), in the free
field against the Fourier symbol and on random gauge fields.  The staggered
operator is pinned by the free-field closed form of D^dagger D on plane
waves, anti-hermiticity of its hopping term, gauge covariance, and the dense
matrix filled from its matrix elements (Schur complement, LU solve).  The
multigrid pieces are pinned to dense linear algebra: P^dag P = 1, the coarse
operator against P^dag M P with the dense matrix-element form M, the block
operator against M with inter-block entries removed, SAP and the cycle
against block Gauss-Seidel half-sweeps written with dense block inverses,
one minimal-residual step against least squares, and the FBiCGStab solve
against LU.
"""

from . import lattice, gamma, dirac, evenodd, domainwall, staggered, multigrid, solvers  # noqa: F401
