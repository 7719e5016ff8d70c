"""Krylov and dense solvers for D x = b.

Sec. 3 of the paper solves the clover system with BiCGStab, compares a
mixed-precision BiCGStab against multigrid, and solves the domain-wall
system with CG (Fig. 7); it prints no solver steps, tolerances or breakdown
handling.  The mixed-precision method reaches the
exact solution of D x = b up to rounding, so the oracle for it is that
solution: a plain FP64 BiCGStab (van der Vorst, 1992) and, on tiny lattices,
a dense LU solve.  Readings taken where the paper is silent:

* <a, b> = sum conj(a) b;  x_0 = 0 unless a guess is given;
* stop when ||r|| <= tol ||b||, then recompute the true residual b - A x and
  continue from it if that is still above tol;
* breakdown (|<r^, r>| < 1e-30 ||r^|| ||r|| or omega = 0): restart from the
  true residual with r^ = r.
"""

from __future__ import annotations

import numpy as np

from . import dirac
from . import gamma as _g
from .lattice import Lattice


def dot(a, b) -> complex:
    return complex(np.vdot(a, b))


def norm(a) -> float:
    return float(np.sqrt(np.vdot(a, a).real))


def bicgstab(A, b, x0=None, tol=1e-12, maxiter=100000):
    """van der Vorst BiCGStab for A x = b; returns (x, info)."""
    bnorm = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    info = {"iters": 0, "restarts": 0, "converged": False, "true_rel_residual": None}
    if bnorm == 0.0:
        info.update(converged=True, true_rel_residual=0.0)
        return np.zeros_like(b), info
    r = b - A(x)
    while info["iters"] < maxiter:
        rhat = r.copy()
        rho = alpha = omega = 1.0 + 0j
        v = np.zeros_like(b)
        p = np.zeros_like(b)
        restart = False
        while info["iters"] < maxiter:
            if norm(r) <= tol * bnorm:
                break
            rho_new = dot(rhat, r)
            if abs(rho_new) < 1e-30 * norm(rhat) * norm(r):
                restart = True
                break
            beta = (rho_new / rho) * (alpha / omega)
            p = r + beta * (p - omega * v)
            v = A(p)
            alpha = rho_new / dot(rhat, v)
            s = r - alpha * v
            t = A(s)
            tt = dot(t, t).real
            omega = dot(t, s) / tt if tt > 0 else 0.0
            x = x + alpha * p + omega * s
            r = s - omega * t
            rho = rho_new
            info["iters"] += 1
            if omega == 0.0:
                restart = True
                break
        r = b - A(x)
        rel = norm(r) / bnorm
        info["true_rel_residual"] = rel
        if rel <= tol:
            info["converged"] = True
            break
        if not restart and info["iters"] >= maxiter:
            break
        info["restarts"] += 1
    return x, info


def cg(A, b, x0=None, tol=1e-12, maxiter=100000):
    """Conjugate gradients (Hestenes-Stiefel) for a Hermitian positive definite A.

    Stops when ||r|| <= tol ||b|| for the recursively updated r, then
    recomputes r = b - A x and restarts from it while that is above tol.
    """
    bnorm = norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    info = {"iters": 0, "restarts": 0, "converged": False, "true_rel_residual": None}
    if bnorm == 0.0:
        info.update(converged=True, true_rel_residual=0.0)
        return np.zeros_like(b), info
    r = b - A(x)
    while info["iters"] < maxiter:
        p = r.copy()
        rr = dot(r, r).real
        while rr > (tol * bnorm) ** 2 and info["iters"] < maxiter:
            Ap = A(p)
            alpha = rr / dot(p, Ap).real
            x = x + alpha * p
            r = r - alpha * Ap
            rr_new = dot(r, r).real
            p = r + (rr_new / rr) * p
            rr = rr_new
            info["iters"] += 1
        r = b - A(x)
        rel = norm(r) / bnorm
        info["true_rel_residual"] = rel
        if rel <= tol:
            info["converged"] = True
            break
        info["restarts"] += 1
    return x, info


def cgnr(D, Ddag, b, tol=1e-12, maxiter=100000):
    """Solve D x = b by CG on the normal equations D^dag D x = D^dag b.

    The stopping test of CG is on the normal residual; the tolerance on it is
    tightened by 10 until the residual of the original system satisfies
    ||b - D x|| <= tol ||b||.
    """
    bnorm = norm(b)
    info = {"iters": 0, "converged": False, "true_rel_residual": 0.0}
    if bnorm == 0.0:
        info["converged"] = True
        return np.zeros_like(b), info
    rhs = Ddag(b)
    x = np.zeros_like(b)
    tn = tol
    while info["iters"] < maxiter:
        x, ci = cg(lambda v: Ddag(D(v)), rhs, x0=x, tol=tn, maxiter=maxiter - info["iters"])
        info["iters"] += ci["iters"]
        rel = norm(b - D(x)) / bnorm
        info["true_rel_residual"] = rel
        if rel <= tol:
            info["converged"] = True
            break
        tn /= 10.0
    return x, info


# --- dense forms (tiny lattices only) -----------------------------------------


def dense_matrix(apply, n: int) -> np.ndarray:
    """Matrix of a linear map on C^n, built column by column from unit vectors."""
    M = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[k] = 1.0
        M[:, k] = apply(e)
    return M


def dense_dirac(U, lat: Lattice, kappa: float, csw: float, bc=(1, 1, 1, -1)) -> np.ndarray:
    """D as a dense (12V x 12V) matrix filled from its matrix elements.

    Row block x, column block y:  T(x) delta_{xy}
      - kappa sum_mu [ bc (1 - gamma_mu) (x) U_mu(x)           if y = x + mu
                     + bc (1 + gamma_mu) (x) U_mu(x - mu)^dag  if y = x - mu ],
    with bc the boundary phase of a wrapping hop.  Written with explicit
    loops over sites, independent of the stencil in ``dirac.hop``.
    """
    V = lat.V
    M = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    T = dirac.clover_term(U, lat, kappa, csw)
    for x in range(V):
        M[12 * x : 12 * x + 12, 12 * x : 12 * x + 12] += T[x]
        for mu in range(4):
            g = _g.GAMMA[mu]
            (y,), (w,) = lat.neighbor(np.array([x]), mu, +1)
            ph = bc[mu] if w else 1.0
            M[12 * x : 12 * x + 12, 12 * y : 12 * y + 12] -= kappa * ph * np.kron(_g.I4 - g, U[mu][x])
            (y,), (w,) = lat.neighbor(np.array([x]), mu, -1)
            ph = bc[mu] if w else 1.0
            M[12 * x : 12 * x + 12, 12 * y : 12 * y + 12] -= kappa * ph * np.kron(_g.I4 + g, U[mu][y].conj().T)
    return M


def lu_solve(M: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Dense solve by LU with partial pivoting (LAPACK gesv)."""
    return np.linalg.solve(M, b)
