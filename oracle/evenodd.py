"""Even-odd blocks and the Schur operator of Eq. 1.

Eq. 1 of the paper writes the full operator in 2x2 block form over even and
odd sites,

    D = [[D_ee, D_eo], [D_oe, D_oo]],   D^(eo) = 1 - D_ee^-1 D_eo D_oo^-1 D_oe,

and uses D^(eo) in the even-odd preconditioned solver.  For D = T - kappa H
the site-local term T is the only part that keeps the parity and H the only
part that flips it, so D_ee = T_e, D_oo = T_o, D_eo = -kappa H_eo and
D_oe = -kappa H_oe.  The solve of D x = b goes through

    b^_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o),   D^(eo) x_e = b^_e,
    x_o  = D_oo^-1 (b_o - D_oe x_e),

which follows from eliminating x_o in the block system (the paper leaves the
source preparation implicit; this is the left-T_ee^-1 form of Eq. 1).
"""

from __future__ import annotations

import numpy as np

from . import dirac
from .lattice import Lattice


class EvenOdd:
    """The blocks of Eq. 1 for one gauge field, kappa, c_sw and boundary."""

    def __init__(self, U, lat: Lattice, kappa: float, csw: float, bc=(1, 1, 1, -1)):
        self.U, self.lat, self.kappa, self.csw, self.bc = U, lat, kappa, csw, tuple(bc)
        self.T = [dirac.clover_term(U, lat, kappa, csw, lat.sites_of(p)) for p in (0, 1)]
        self.Tinv = [np.linalg.inv(t) for t in self.T]

    # --- the four blocks -------------------------------------------------
    def D_pp(self, parity: int, v):
        """D_ee (parity 0) or D_oo (parity 1): the site-local term T."""
        return dirac.apply_site(self.T[parity], v)

    def D_pp_inv(self, parity: int, v):
        return dirac.apply_site(self.Tinv[parity], v)

    def D_hop(self, out_parity: int, v):
        """D_eo (out_parity 0, v odd) or D_oe (out_parity 1, v even): -kappa H."""
        lat = self.lat
        full = lat.embed(v, 1 - out_parity)
        return -self.kappa * dirac.hop(self.U, full, lat, self.bc, lat.sites_of(out_parity))

    # --- Eq. 1 ---------------------------------------------------------------
    def schur(self, x_e):
        """D^(eo) x_e = x_e - D_ee^-1 D_eo D_oo^-1 D_oe x_e."""
        t = self.D_pp_inv(1, self.D_hop(1, x_e))
        return x_e - self.D_pp_inv(0, self.D_hop(0, t))

    def prepare(self, b):
        """b^_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o) from a full-lattice source b."""
        lat = self.lat
        b_e, b_o = b[lat.even], b[lat.odd]
        return self.D_pp_inv(0, b_e - self.D_hop(0, self.D_pp_inv(1, b_o)))

    def reconstruct(self, x_e, b):
        """Full solution from x_e: x_o = D_oo^-1 (b_o - D_oe x_e)."""
        lat = self.lat
        x = np.zeros((lat.V, 4, 3), dtype=np.complex128)
        x[lat.even] = x_e
        x[lat.odd] = self.D_pp_inv(1, b[lat.odd] - self.D_hop(1, x_e))
        return x

    def full(self, psi):
        """The full operator assembled from the blocks (for cross-checks)."""
        lat = self.lat
        out = np.zeros_like(psi)
        for p in (0, 1):
            s = lat.sites_of(p)
            out[s] = self.D_pp(p, psi[s]) + self.D_hop(p, psi[lat.sites_of(1 - p)])
        return out
