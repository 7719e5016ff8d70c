"""Gamma matrices for the Wilson/clover operator.

The paper (Sec. 2) states only that its layout follows the QWS gamma
convention with gamma_5 of opposite sign and that data is converted at the
call boundary; it prints no basis.  Reading taken: the chiral basis

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = 1, 2, 3 -> x, y, z)
    gamma_4 = [[0, 1], [1, 0]]                     (t)

so that gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1) and
sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] is block diagonal in spin.
Index mu = 0, 1, 2, 3 means x, y, z, t.
"""

from __future__ import annotations

import numpy as np

PAULI = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]

I2 = np.eye(2, dtype=np.complex128)
Z2 = np.zeros((2, 2), dtype=np.complex128)
I4 = np.eye(4, dtype=np.complex128)


def _build():
    g = [np.block([[Z2, -1j * PAULI[k]], [1j * PAULI[k], Z2]]) for k in range(3)]
    g.append(np.block([[Z2, I2], [I2, Z2]]))
    return g


GAMMA = _build()


def gamma5() -> np.ndarray:
    return GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def sigma(mu: int, nu: int) -> np.ndarray:
    """sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu]."""
    return 0.5j * (GAMMA[mu] @ GAMMA[nu] - GAMMA[nu] @ GAMMA[mu])
