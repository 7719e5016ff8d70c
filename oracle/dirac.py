"""Wilson and clover Dirac operators, written out from their definitions.

The paper (Sec. 2) implements the Wilson and clover (Sheikholeslami-Wohlert)
fermion operators and their even-odd blocks; it prints no operator formula
beyond the even-odd decomposition of Eq. 1.  Readings taken (the standard
textbook forms):

* hopping term
      (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                          + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ],
  with the boundary phase bc[mu] on every hop that wraps around the lattice;
* Wilson operator D_W = 1 - kappa H;
* clover operator D = T - kappa H with the site-local term
      T(x) = 1 - kappa c_sw sum_{mu < nu} sigma_{mu nu} F_{mu nu}(x),
      F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / (8 i), made traceless,
  where Q_{mu nu}(x) is the sum of the four plaquettes in the (mu, nu) plane
  that have a corner at x, each run counter-clockwise starting at x.

Everything is vectorised over a list of sites with numpy; nothing is blocked
or fused.  ``sites=None`` means all sites.
"""

from __future__ import annotations

import numpy as np

from . import gamma as _g
from .lattice import Lattice


def _dag(A: np.ndarray) -> np.ndarray:
    return np.conj(np.swapaxes(A, -1, -2))


def _spin(P: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to spinors of shape (n, 4, 3)."""
    return np.einsum("st,ntc->nsc", P, chi)


def _colour(U: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """Apply 3x3 colour matrices U (n, 3, 3) to spinors chi (n, 4, 3)."""
    return chi @ np.swapaxes(U, -1, -2)


def hop(U, psi, lat: Lattice, bc=(1, 1, 1, -1), sites=None) -> np.ndarray:
    """(H psi)(x) for x in ``sites``."""
    if sites is None:
        sites = np.arange(lat.V)
    out = np.zeros((len(sites), 4, 3), dtype=np.complex128)
    for mu in range(4):
        g = _g.GAMMA[mu]
        # forward hop: (1 - gamma_mu) U_mu(x) psi(x + mu)
        j, wraps = lat.neighbor(sites, mu, +1)
        phase = np.where(wraps, bc[mu], 1.0)[:, None, None]
        out += _spin(_g.I4 - g, _colour(U[mu][sites], phase * psi[j]))
        # backward hop: (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu)
        j, wraps = lat.neighbor(sites, mu, -1)
        phase = np.where(wraps, bc[mu], 1.0)[:, None, None]
        out += _spin(_g.I4 + g, _colour(_dag(U[mu][j]), phase * psi[j]))
    return out


def wilson(U, psi, lat: Lattice, kappa: float, bc=(1, 1, 1, -1), sites=None) -> np.ndarray:
    """D_W psi = psi - kappa H psi at ``sites``."""
    if sites is None:
        sites = np.arange(lat.V)
    return psi[sites] - kappa * hop(U, psi, lat, bc, sites)


def clover_leaves(U, lat: Lattice, sites, mu: int, nu: int) -> np.ndarray:
    """Q_{mu nu}(x): sum of the four counter-clockwise plaquettes at x."""
    x = sites
    xpm, _ = lat.neighbor(x, mu, +1)
    xpn, _ = lat.neighbor(x, nu, +1)
    xmm, _ = lat.neighbor(x, mu, -1)
    xmn, _ = lat.neighbor(x, nu, -1)
    xmm_pn, _ = lat.neighbor(xmm, nu, +1)
    xmm_mn, _ = lat.neighbor(xmm, nu, -1)
    xpm_mn, _ = lat.neighbor(xpm, nu, -1)
    Um, Un = U[mu], U[nu]
    q = Um[x] @ Un[xpm] @ _dag(Um[xpn]) @ _dag(Un[x])
    q = q + Un[x] @ _dag(Um[xmm_pn]) @ _dag(Un[xmm]) @ Um[xmm]
    q = q + _dag(Um[xmm]) @ _dag(Un[xmm_mn]) @ Um[xmm_mn] @ Un[xmn]
    q = q + _dag(Un[xmn]) @ Um[xmn] @ Un[xpm_mn] @ _dag(Um[x])
    return q


def field_strength(U, lat: Lattice, sites, mu: int, nu: int) -> np.ndarray:
    """F_{mu nu}(x) = (Q - Q^dagger)/(8i) minus its trace over 3."""
    Q = clover_leaves(U, lat, sites, mu, nu)
    F = (Q - _dag(Q)) / 8j
    tr = np.trace(F, axis1=-2, axis2=-1)
    return F - (tr / 3.0)[:, None, None] * np.eye(3)


def clover_term(U, lat: Lattice, kappa: float, csw: float, sites=None) -> np.ndarray:
    """T(x) as 12x12 matrices (index spin*3 + colour), shape (n, 12, 12)."""
    if sites is None:
        sites = np.arange(lat.V)
    n = len(sites)
    T = np.broadcast_to(np.eye(12, dtype=np.complex128), (n, 12, 12)).copy()
    if csw == 0.0 or kappa == 0.0:
        return T
    for mu in range(4):
        for nu in range(mu + 1, 4):
            F = field_strength(U, lat, sites, mu, nu)
            S = _g.sigma(mu, nu)
            T -= kappa * csw * np.einsum("st,nab->nsatb", S, F).reshape(n, 12, 12)
    return T


def apply_site(M: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Site-local 12x12 matrices M (n, 12, 12) times spinors psi (n, 4, 3)."""
    return (M @ psi.reshape(-1, 12, 1)).reshape(-1, 4, 3)


def dirac(U, psi, lat: Lattice, kappa: float, csw: float, bc=(1, 1, 1, -1), sites=None, T=None) -> np.ndarray:
    """Full operator D psi = T psi - kappa H psi at ``sites`` (T = 1 for c_sw = 0).

    ``T`` may be passed precomputed for the same ``sites``.
    """
    if sites is None:
        sites = np.arange(lat.V)
    if T is None:
        T = clover_term(U, lat, kappa, csw, sites)
    return apply_site(T, psi[sites]) - kappa * hop(U, psi, lat, bc, sites)


def plaquette(U, lat: Lattice) -> float:
    """Average of Re tr P_{mu nu}(x) / 3 over sites and the six planes."""
    x = np.arange(lat.V)
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            xpm, _ = lat.neighbor(x, mu, +1)
            xpn, _ = lat.neighbor(x, nu, +1)
            P = U[mu][x] @ U[nu][xpm] @ _dag(U[mu][xpn]) @ _dag(U[nu][x])
            acc += np.trace(P, axis1=-2, axis2=-1).real.sum()
    return acc / (6 * 3 * lat.V)
