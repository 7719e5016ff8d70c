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
import os
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
    """n traceless Hermitian matrices A = sum_a w_a l_a / 2 with w_a ~ N(0, 1), shape (n, 3, 3)."""
    w = gen.standard_normal((n, 8))
    return np.einsum("na,aij->nij", w, GELL_MANN) * 0.5


def _mm(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Products of 3x3 matrices stored component-major, shape (3, 3, n)."""
    return np.einsum("ikn,kjn->ijn", A, B)


def _expi_soa(A: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*A) for Hermitian A in component-major form (3, 3, n).

    Scaling and squaring: the argument is scaled to Frobenius norm <= 1/8,
    where the degree-12 Taylor polynomial (Horner form) is exact to far below
    1e-18, then squared back.
    """
    X = 1j * float(eps) * A
    n = X.shape[-1]
    if n == 0:
        return X
    nrm = float(np.sqrt(np.max(np.sum(np.abs(X) ** 2, axis=(0, 1)))))
    s = max(0, int(math.ceil(math.log2(nrm / 0.125)))) if nrm > 0.125 else 0
    X = X / (2.0**s)
    eye = np.zeros_like(X)
    for k in range(3):
        eye[k, k] = 1.0
    E = eye.copy()
    for k in range(12, 0, -1):  # I + X/1 (I + X/2 (I + ...))
        E = eye + _mm(X, E) / k
    for _ in range(s):
        E = _mm(E, E)
    return E


def _reunitarize_soa(U: np.ndarray) -> np.ndarray:
    """Project (3, 3, n) matrices onto SU(3): Gram-Schmidt rows 1, 2; row 3 = conj(r1 x r2)."""
    r1 = U[0] / np.sqrt(np.sum(np.abs(U[0]) ** 2, axis=0))
    r2 = U[1] - np.sum(r1.conj() * U[1], axis=0) * r1
    r2 = r2 / np.sqrt(np.sum(np.abs(r2) ** 2, axis=0))
    r3 = np.stack(
        [r1[1] * r2[2] - r1[2] * r2[1], r1[2] * r2[0] - r1[0] * r2[2], r1[0] * r2[1] - r1[1] * r2[0]]
    ).conj()
    return np.stack([r1, r2, r3])


def expi_hermitian(A: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*A) for a batch of Hermitian A of shape (n, 3, 3)."""
    return np.ascontiguousarray(_expi_soa(np.transpose(A, (1, 2, 0)), eps).transpose(2, 0, 1))


def reunitarize(U: np.ndarray) -> np.ndarray:
    """Project a batch (n, 3, 3) onto SU(3): Gram-Schmidt rows 1, 2; row 3 = conj(r1 x r2)."""
    return np.ascontiguousarray(_reunitarize_soa(np.transpose(U, (1, 2, 0))).transpose(2, 0, 1))


def gauge_field(dims, eps: float, seed: int, chunk: int = 1 << 18, threads: int | None = None) -> np.ndarray:
    """Links U_mu(x) = exp(i*eps*A_mu(x)), shape (4, V, 3, 3), complex128.

    The Lie-algebra draws are taken chunk by chunk in a fixed order from one
    PCG64 stream; only the exponentiation runs on a thread pool, so the field
    does not depend on the thread count.
    """
    from concurrent.futures import ThreadPoolExecutor

    V = volume(dims)
    n = 4 * V
    gen = rng(seed, FIELD_GAUGE)
    out = np.empty((n, 3, 3), dtype=np.complex128)

    def work(lo, w):
        A = np.einsum("an,aij->ijn", w.T, GELL_MANN) * 0.5
        out[lo : lo + w.shape[0]] = _reunitarize_soa(_expi_soa(A, eps)).transpose(2, 0, 1)

    nt = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(max_workers=nt) as ex:
        futs = []
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            futs.append(ex.submit(work, lo, gen.standard_normal((hi - lo, 8))))
            if len(futs) >= 2 * nt:
                futs.pop(0).result()
        for f in futs:
            f.result()
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
    return gen.standard_normal(shape + (2,)).view(np.complex128)[..., 0]


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
    inner: str = "f32"  # storage precision of the inner solver

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
    # Mid-size clover case (working set above L2, a few GB) for profiler captures.
    "clover_24x24x24x48": Workload("clover_24x24x24x48", (24, 24, 24, 48), "clover", 0.125, 1.0, 0.2, 4, 1, "gaussian", 1e-10),
    # The same with twelve point sources, for profiler captures of the multi-RHS kernels.
    "clover_24x24x24x48_12rhs": Workload(
        "clover_24x24x24x48_12rhs", (24, 24, 24, 48), "clover", 0.125, 1.0, 0.2, 4, 12, "point", 1e-10, inner="f16"
    ),
    # The 32^3x64 clover field near its critical kappa (BiCGStab needs ~500
    # iterations): the multigrid solver's workload.
    "mg_clover_32x32x32x64": Workload("mg_clover_32x32x32x64", (32, 32, 32, 64), "clover", 0.1275, 1.0, 0.2, 2, 1, "gaussian", 1e-10),
    # Twelve point sources on 48^3x96 clover with half-precision storage.
    "clover_48x48x48x96_12rhs": Workload(
        "clover_48x48x48x96_12rhs", (48, 48, 48, 96), "clover", 0.125, 1.0, 0.2, 3, 12, "point", 1e-10, inner="f16"
    ),
}


@dataclass(frozen=True)
class MobiusWorkload:
    """One synthetic configuration of the Moebius domain-wall solver path."""

    name: str
    dims: tuple
    Ls: int
    M5: float
    b5: float
    c5: float
    mf: float
    eps: float
    seed: int
    nrhs: int
    tol: float
    bc: tuple = field(default=(1, 1, 1, -1))
    inner: str = "f32"
    kind: str = "mobius"

    @property
    def volume(self) -> int:
        return volume(self.dims)

    def gauge(self) -> np.ndarray:
        return gauge_field(self.dims, self.eps, self.seed)

    def sources(self) -> np.ndarray:
        """Gaussian five-dimensional sources shaped (nrhs, Ls, V, 4, 3)."""
        b = gaussian_spinor(self.dims, self.seed, nrhs=self.nrhs * self.Ls)
        return b.reshape((self.nrhs, self.Ls) + b.shape[1:])


# Moebius domain wall on 24^3x48 with Ls = 16, M5 = 1.8, b = 1.5, c = 0.5,
# m_f = 0.01: CG on the normal equations, FP32 inner / FP64 outer to 1e-10.
WORKLOADS["mobius_24x24x24x48x16"] = MobiusWorkload(
    "mobius_24x24x24x48x16", (24, 24, 24, 48), 16, 1.8, 1.5, 0.5, 0.01, 0.2, 5, 1, 1e-10
)
# The same on 16^3x32 (each five-dimensional FP32 field 201 MB, above L2; a
# few GB in all) for profiler captures.
WORKLOADS["mobius_16x16x16x32x16"] = MobiusWorkload(
    "mobius_16x16x16x32x16", (16, 16, 16, 32), 16, 1.8, 1.5, 0.5, 0.01, 0.2, 5, 1, 1e-10
)


@dataclass(frozen=True)
class StaggeredWorkload:
    """One synthetic configuration of the staggered solver path."""

    name: str
    dims: tuple
    mass: float
    eps: float
    seed: int
    nrhs: int
    tol: float
    bc: tuple = field(default=(1, 1, 1, -1))
    inner: str = "f32"
    kind: str = "staggered"

    @property
    def volume(self) -> int:
        return volume(self.dims)

    def gauge(self) -> np.ndarray:
        return gauge_field(self.dims, self.eps, self.seed)

    def sources(self) -> np.ndarray:
        """Gaussian colour-vector sources shaped (nrhs, V, 3)."""
        V = volume(self.dims)
        gen = rng(self.seed, FIELD_SOURCE)
        return gen.standard_normal((self.nrhs, V, 3, 2)).view(np.complex128)[..., 0]


# Staggered on 64^4, m = 0.05, links exp(0.2 i A): CG on the even system,
# FP32 inner / FP64 outer to 1e-10.
WORKLOADS["staggered_64x64x64x64"] = StaggeredWorkload("staggered_64x64x64x64", (64, 64, 64, 64), 0.05, 0.2, 6, 1, 1e-10)
# The same on 32^4 (links above L2, a few GB in all) for profiler captures.
WORKLOADS["staggered_32x32x32x32"] = StaggeredWorkload("staggered_32x32x32x32", (32, 32, 32, 32), 0.05, 0.2, 6, 1, 1e-10)
