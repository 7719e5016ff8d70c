"""Staggered fermion operator and its even-odd blocks.

The paper (Sec. 2) implements the standard staggered action beside
Wilson/clover and domain wall, with even-odd versions in the block form of
Eq. 1; it prints no formula.  Readings taken (the textbook Kogut-Susskind
operator):

* one colour vector chi(x) (3 complex numbers) per site;
* staggered phases eta_0(x) = 1, eta_1(x) = (-1)^x0, eta_2(x) = (-1)^(x0+x1),
  eta_3(x) = (-1)^(x0+x1+x2), with (x0, x1, x2, x3) = (x, y, z, t);
* D chi(x) = m chi(x) + (1/2) sum_mu eta_mu(x) [ U_mu(x) chi(x + mu)
                                               - U_mu(x - mu)^dagger chi(x - mu) ],
  with the boundary phase bc[mu] on every hop that wraps (as for Wilson).

The hopping part is anti-Hermitian, so with D_ee = D_oo = m and D_eo, D_oe
the hopping blocks, the Schur operator of Eq. 1 is
D^(eo) = 1 - D_eo D_oe / m^2 = (m^2 - D_eo D_oe) / m^2, and m^2 - D_eo D_oe
is Hermitian positive definite: it is the even-even block of D^dagger D.  The
solve runs CG on (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o (that block of the
normal equations) and reconstructs x_o = (b_o - D_oe x_e) / m.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import numpy as np

from .lattice import Lattice


def _dag(A):
    return np.conj(np.swapaxes(A, -1, -2))


def eta(lat: Lattice, mu: int) -> np.ndarray:
    """Staggered phase eta_mu(x) at every site."""
    s = np.zeros(lat.V, dtype=np.int64)
    for nu in range(mu):
        s = s + lat.coords[nu]
    return np.where(s % 2 == 0, 1.0, -1.0)


def hop(U, chi, lat: Lattice, bc=(1, 1, 1, -1), sites=None) -> np.ndarray:
    """(1/2) sum_mu eta_mu(x) [U_mu(x) chi(x+mu) - U_mu(x-mu)^dag chi(x-mu)] at ``sites``."""
    if sites is None:
        sites = np.arange(lat.V)
    out = np.zeros((len(sites), 3), dtype=np.complex128)
    for mu in range(4):
        e = eta(lat, mu)[sites][:, None]
        j, wraps = lat.neighbor(sites, mu, +1)
        ph = np.where(wraps, bc[mu], 1.0)[:, None]
        out += 0.5 * e * np.einsum("nab,nb->na", U[mu][sites], ph * chi[j])
        j, wraps = lat.neighbor(sites, mu, -1)
        ph = np.where(wraps, bc[mu], 1.0)[:, None]
        out -= 0.5 * e * np.einsum("nab,nb->na", _dag(U[mu][j]), ph * chi[j])
    return out


class Staggered:
    """Staggered operator for one gauge field, mass and boundary."""

    def __init__(self, U, lat: Lattice, mass: float, bc=(1, 1, 1, -1)):
        self.U, self.lat, self.m, self.bc = U, lat, float(mass), tuple(bc)

    def full(self, chi, sites=None):
        """D chi = m chi + hop chi, chi of shape (V, 3)."""
        if sites is None:
            sites = np.arange(self.lat.V)
        return self.m * chi[sites] + hop(self.U, chi, self.lat, self.bc, sites)

    def D_hop(self, out_parity: int, v):
        """D_eo (out_parity 0, v odd) or D_oe (1, v even) on half-lattice vectors (V/2, 3)."""
        lat = self.lat
        return hop(self.U, lat.embed(v, 1 - out_parity), lat, self.bc, lat.sites_of(out_parity))

    def schur(self, x_e):
        """D^(eo) x_e = x_e - D_eo D_oe x_e / m^2 (Eq. 1 with D_ee = D_oo = m)."""
        return x_e - self.D_hop(0, self.D_hop(1, x_e)) / self.m**2

    def normal_even(self, x_e):
        """(m^2 - D_eo D_oe) x_e, the even-even block of D^dagger D."""
        return self.m**2 * x_e - self.D_hop(0, self.D_hop(1, x_e))

    def prepare(self, b):
        """Right-hand side of the even system: m b_e - D_eo b_o."""
        lat = self.lat
        return self.m * b[lat.even] - self.D_hop(0, b[lat.odd])

    def reconstruct(self, x_e, b):
        """Full solution: x_o = (b_o - D_oe x_e) / m."""
        lat = self.lat
        x = np.zeros((lat.V, 3), dtype=np.complex128)
        x[lat.even] = x_e
        x[lat.odd] = (b[lat.odd] - self.D_hop(1, x_e)) / self.m
        return x
