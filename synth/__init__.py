"""Seeded synthetic inputs for the Wilson/clover solver path.

This module produces the inputs that both the FP64 CPU oracle and the CUDA
library consume: SU(3) gauge fields U = exp(i*eps*A) with A a Gaussian
traceless Hermitian 3x3 matrix per link, Gaussian complex spinor sources and
point sources.  It holds none of the Dirac-operator or solver arithmetic; it
only draws random numbers and exponentiates Lie-algebra elements, so that the
same seeded input can be handed to both sides of a parity test.

Conventions (canonical host layouts, shared by every caller):

* lattice extents ``dims = (Lx, Ly, Lz, Lt)``; lexicographic site index
  ``i = x + Lx*(y + Ly*(z + Lz*t))`` (x fastest);
* spinor fields: complex128 arrays of shape ``(V, 4, 3)`` or
  ``(nrhs, V, 4, 3)`` -- [rhs][t][z][y][x][spin][colour] with (re, im) pairs
  when viewed as float64;
* gauge fields: complex128 arrays of shape ``(4, V, 3, 3)`` --
  [mu][t][z][y][x][row][col], mu = x, y, z, t.

Every draw uses a PCG64 stream keyed by ``(seed, field_id)`` so that the gauge
field and the sources of one configuration are independent and reproducible.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "GELL_MANN",
    "volume",
    "rng",
    "lie_gaussian",
    "expi_hermitian",
    "reunitarize",
    "gauge_field",
    "unit_gauge",
    "gaussian_spinor",
    "point_sources",
    "Workload",
    "WORKLOADS",
]

# Field ids for the PCG64 streams of one configuration.
FIELD_GAUGE = 0
FIELD_SOURCE = 1
FIELD_AUX = 2


def _gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, normalised tr(l_a l_b) = 2 delta_ab."""
    g = np.zeros((8, 3, 3), dtype=np.complex128)
    g[0][0, 1] = g[0][1, 0] = 1
    g[1][0, 1] = -1j
    g[1][1, 0] = 1j
    g[2][0, 0] = 1
    g[2][1, 1] = -1
    g[3][0, 2] = g[3][2, 0] = 1
    g[4][0, 2] = -1j
    g[4][2, 0] = 1j
    g[5][1, 2] = g[5][2, 1] = 1
    g[6][1, 2] = -1j
    g[6][2, 1] = 1j
    g[7][0, 0] = g[7][1, 1] = 1 / math.sqrt(3)
    g[7][2, 2] = -2 / math.sqrt(3)
    return g


GELL_MANN = _gell_mann()


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def rng(seed: int, field_id: int) -> np.random.Generator:
    """PCG64 stream for one (configuration seed, field) pair."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(field_id)])))


def lie_gaussian(gen: np.random.Generator, n: int) -> np.ndarray:
    """n traceless Hermitian matrices A = sum_a w_a l_a / 2 with w_a ~ N(0, 1)."""
    w = gen.standard_normal((n, 8))
    return np.einsum("na,aij->nij", w, GELL_MANN) * 0.5


def expi_hermitian(A: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*A) for a batch of Hermitian A by scaling and squaring.

    The scaled argument has Frobenius norm <= 1/2, where the degree-16
    Taylor polynomial is exact to below 1e-19; the result is squared back.
    """
    X = 1j * float(eps) * A
    nrm = float(np.max(np.sqrt(np.sum(np.abs(X) ** 2, axis=(-2, -1))))) if len(X) else 0.0
    s = max(0, int(math.ceil(math.log2(nrm / 0.5)))) if nrm > 0.5 else 0
    X = X / (2.0**s)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), X.shape)
    E = eye.copy()
    for k in range(16, 0, -1):  # Horner: I + X/1 (I + X/2 (I + ...))
        E = eye + (X @ E) / k
    for _ in range(s):
        E = E @ E
    return E


def reunitarize(U: np.ndarray) -> np.ndarray:
    """Project onto SU(3): Gram-Schmidt on rows 1, 2; row 3 = conj(r1 x r2)."""
    r1 = U[..., 0, :]
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = U[..., 1, :]
    r2 = r2 - np.sum(r1.conj() * r2, axis=-1, keepdims=True) * r1
    r2 = r2 / np.linalg.norm(r2, axis=-1, keepdims=True)
    r3 = np.cross(r1, r2).conj()
    return np.stack([r1, r2, r3], axis=-2)


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    """Links U_mu(x) = exp(i*eps*A_mu(x)), shape (4, V, 3, 3), complex128."""
    V = volume(dims)
    n = 4 * V
    gen = rng(seed, FIELD_GAUGE)
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for lo in range(0, n, chunk):
        hi = min(n, lo + chunk)
        A = lie_gaussian(gen, hi - lo)
        out[lo:hi] = reunitarize(expi_hermitian(A, eps))
    return out.reshape(4, V, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    V = volume(dims)
    U = np.zeros((4, V, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    return U


def gaussian_spinor(dims, seed: int, nrhs: int | None = None, field_id: int = FIELD_SOURCE) -> np.ndarray:
    """Spinor(s) whose real and imaginary parts are each N(0, 1)."""
    V = volume(dims)
    shape = (V, 4, 3) if nrhs is None else (nrhs, V, 4, 3)
    gen = rng(seed, field_id)
    re = gen.standard_normal(shape)
    im = gen.standard_normal(shape)
    return re + 1j * im


def point_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, shape (12, V, 4, 3)."""
    V = volume(dims)
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        b[k, site, k // 3, k % 3] = 1
    return b


@dataclass(frozen=True)
class Workload:
    """One synthetic configuration of the solver path."""

    name: str
    dims: tuple
    kind: str  # "wilson" or "clover"
    kappa: float
    csw: float
    eps: float
    seed: int
    nrhs: int
    source: str  # "gaussian" or "point"
    tol: float
    bc: tuple = field(default=(1, 1, 1, -1))

    @property
    def volume(self) -> int:
        return volume(self.dims)

    def gauge(self) -> np.ndarray:
        return gauge_field(self.dims, self.eps, self.seed)

    def sources(self) -> np.ndarray:
        """Sources shaped (nrhs, V, 4, 3)."""
        if self.source == "point":
            return point_sources(self.dims)[: self.nrhs]
        return gaussian_spinor(self.dims, self.seed, nrhs=self.nrhs)


WORKLOADS = {
    # Wilson D on 8^4, FP64, apply and solve to 1e-12 (correctness case; fits in L2).
    "wilson_8x8x8x8": Workload("wilson_8x8x8x8", (8, 8, 8, 8), "wilson", 0.12, 0.0, 0.3, 1, 1, "gaussian", 1e-12),
    # Even-odd clover on 32^3x64: FP32 inner BiCGStab + FP64 defect correction vs plain FP64.
    "clover_32x32x32x64": Workload("clover_32x32x32x64", (32, 32, 32, 64), "clover", 0.125, 1.0, 0.2, 2, 1, "gaussian", 1e-10),
    # Twelve point sources on 48^3x96 clover with half-precision storage.
    "clover_48x48x48x96_12rhs": Workload(
        "clover_48x48x48x96_12rhs", (48, 48, 48, 96), "clover", 0.125, 1.0, 0.2, 3, 12, "point", 1e-10
    ),
}
