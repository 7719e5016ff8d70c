"""Moebius domain-wall operator, its even-odd blocks and their adjoints.

The paper (Sec. 2) implements the Moebius domain-wall action beside
Wilson/clover, with even-odd versions of every operator in the block form of
Eq. 1, and a variant that keeps the fifth coordinate s as an inner degree of
freedom of each four-dimensional site; its solver for this operator is CG
(Sec. 3, Fig. 7).  It prints no formula.  Readings taken (the standard
Moebius form of Brower, Neff and Orginos, with constant b, c):

* fields psi[s, x, spin, colour], s = 0 .. Ls-1, x a four-dimensional site;
* the kernel W = D_W(-M5) = (4 - M5) - H/2, with H the Wilson hopping term
  (boundary phases as for Wilson);
* P_+- = (1 +- gamma_5)/2 and the fifth-direction hop
      (P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
  with psi_{Ls} -> -m_f psi_0 and psi_{-1} -> -m_f psi_{Ls-1};
* D psi = (b W + 1) psi + (c W - 1) P psi
  (b = 1, c = 0 is the Shamir operator).

Even-odd split by the parity of the four-dimensional site x (s does not
enter): with alpha = 4 - M5 and the site-local matrices
      A = (b alpha + 1) + (c alpha - 1) P,     B = b + c P,
acting on s and spin only, D_ee = D_oo = A and D_eo, D_oe = -(1/2) H_eo B,
-(1/2) H_oe B (B acts first).  A and B are block diagonal in chirality: on
the P_+ components they are real Ls x Ls matrices built from the shift
s -> s-1, on the P_- components from s -> s+1.

Adjoints use (H_eo)^dagger = gamma_5 H_oe gamma_5 (gamma_5-hermiticity of
the Wilson hopping term) and real transposes for the s-matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import numpy as np

from . import dirac
from .lattice import Lattice

UPPER = slice(0, 2)  # P_+ components in the chiral basis (gamma_5 = diag(1, 1, -1, -1))
LOWER = slice(2, 4)  # P_- components


def shift_matrix(Ls: int, chirality: int, mf: float) -> np.ndarray:
    """The s-part of P on one chirality: (S psi)_s = psi_{s-1} for P_+ (chirality +1),
    psi_{s+1} for P_- (chirality -1), with the -m_f wrap."""
    S = np.zeros((Ls, Ls))
    for s in range(Ls):
        if chirality > 0:
            if s >= 1:
                S[s, s - 1] = 1.0
            else:
                S[s, Ls - 1] = -mf
        else:
            if s + 1 < Ls:
                S[s, s + 1] = 1.0
            else:
                S[s, 0] = -mf
    return S


def _mix(M_plus, M_minus, v):
    """Apply real s-matrices per chirality: v[s, n, spin, colour]."""
    out = np.empty_like(v)
    out[:, :, UPPER] = np.einsum("st,tnac->snac", M_plus, v[:, :, UPPER])
    out[:, :, LOWER] = np.einsum("st,tnac->snac", M_minus, v[:, :, LOWER])
    return out


def _g5(v):
    out = v.copy()
    out[:, :, LOWER] *= -1.0
    return out


class Mobius:
    """Moebius domain-wall operator for one gauge field and parameter set."""

    def __init__(self, U, lat: Lattice, Ls: int, M5: float, b: float, c: float, mf: float, bc=(1, 1, 1, -1)):
        self.U, self.lat, self.Ls = U, lat, int(Ls)
        self.M5, self.b, self.c, self.mf, self.bc = M5, b, c, mf, tuple(bc)
        alpha = 4.0 - M5
        I = np.eye(self.Ls)
        Sp, Sm = shift_matrix(self.Ls, +1, mf), shift_matrix(self.Ls, -1, mf)
        self.A = [(b * alpha + 1) * I + (c * alpha - 1) * Sp, (b * alpha + 1) * I + (c * alpha - 1) * Sm]
        self.B = [b * I + c * Sp, b * I + c * Sm]
        self.Ainv = [np.linalg.inv(a) for a in self.A]

    # --- the full operator, from its definition --------------------------------
    def W(self, psi4, sites=None):
        """D_W(-M5) psi = (4 - M5) psi - H psi / 2 on one slice (V, 4, 3)."""
        lat = self.lat
        if sites is None:
            sites = np.arange(lat.V)
        return (4.0 - self.M5) * psi4[sites] - 0.5 * dirac.hop(self.U, psi4, lat, self.bc, sites)

    def s_hop(self, psi):
        """(P psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}, wraps with -m_f."""
        Ls, mf = self.Ls, self.mf
        out = np.zeros_like(psi)
        for s in range(Ls):
            up = psi[s + 1] if s + 1 < Ls else -mf * psi[0]
            dn = psi[s - 1] if s >= 1 else -mf * psi[Ls - 1]
            out[s][:, LOWER] = up[:, LOWER]
            out[s][:, UPPER] = dn[:, UPPER]
        return out

    def full(self, psi, sites=None):
        """D psi = (b W + 1) psi + (c W - 1) P psi, psi of shape (Ls, V, 4, 3)."""
        if sites is None:
            sites = np.arange(self.lat.V)
        Ppsi = self.s_hop(psi)
        return np.stack(
            [self.b * self.W(psi[s], sites) + psi[s][sites] + self.c * self.W(Ppsi[s], sites) - Ppsi[s][sites]
             for s in range(self.Ls)]
        )

    # --- even-odd blocks (Eq. 1) -----------------------------------------------
    def D_pp(self, v):
        """D_ee = D_oo = A on half-lattice vectors (Ls, V/2, 4, 3)."""
        return _mix(self.A[0], self.A[1], v)

    def D_pp_inv(self, v):
        return _mix(self.Ainv[0], self.Ainv[1], v)

    def D_hop(self, out_parity: int, v):
        """D_eo (out_parity 0, v odd) or D_oe (1, v even): -(1/2) H (B v)."""
        lat = self.lat
        Bv = _mix(self.B[0], self.B[1], v)
        out = np.empty_like(v)
        for s in range(self.Ls):
            full = lat.embed(Bv[s], 1 - out_parity)
            out[s] = -0.5 * dirac.hop(self.U, full, lat, self.bc, lat.sites_of(out_parity))
        return out

    def schur(self, x_e):
        """D^(eo) x_e = x_e - D_ee^-1 D_eo D_oo^-1 D_oe x_e."""
        t = self.D_pp_inv(self.D_hop(1, x_e))
        return x_e - self.D_pp_inv(self.D_hop(0, t))

    def prepare(self, b):
        """b^_e = D_ee^-1 (b_e - D_eo D_oo^-1 b_o) from a full 5-d source (Ls, V, 4, 3)."""
        lat = self.lat
        return self.D_pp_inv(b[:, lat.even] - self.D_hop(0, self.D_pp_inv(b[:, lat.odd])))

    def reconstruct(self, x_e, b):
        """Full solution from x_e: x_o = D_oo^-1 (b_o - D_oe x_e)."""
        lat = self.lat
        x = np.zeros((self.Ls, lat.V, 4, 3), dtype=np.complex128)
        x[:, lat.even] = x_e
        x[:, lat.odd] = self.D_pp_inv(b[:, lat.odd] - self.D_hop(1, x_e))
        return x

    # --- adjoints --------------------------------------------------------------
    def D_pp_inv_dag(self, v):
        return _mix(self.Ainv[0].T, self.Ainv[1].T, v)

    def D_hop_dag(self, in_parity: int, v):
        """(D_{p, 1-p})^dagger v for v on parity p = in_parity, result on 1 - p:
        -(1/2) B^T gamma_5 H_{1-p, p} gamma_5 v."""
        lat = self.lat
        g5v = _g5(v)
        h = np.empty_like(v)
        for s in range(self.Ls):
            full = lat.embed(g5v[s], in_parity)
            h[s] = -0.5 * dirac.hop(self.U, full, lat, self.bc, lat.sites_of(1 - in_parity))
        return _mix(self.B[0].T, self.B[1].T, _g5(h))

    def schur_dag(self, y_e):
        """(D^(eo))^dagger y_e = y_e - D_oe^dag D_oo^-dag D_eo^dag D_ee^-dag y_e."""
        t = self.D_pp_inv_dag(self.D_hop_dag(0, self.D_pp_inv_dag(y_e)))
        return y_e - self.D_hop_dag(1, t)
