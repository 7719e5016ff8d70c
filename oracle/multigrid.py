"""Two-level multigrid for the clover operator: aggregation, P^dag D P, SAP and FBiCGStab.

Sec. 3 of the paper benchmarks a two-level variant of DD-alpha-AMG for the
clover operator: an outer Flexible BiCGStab preconditioned by a
single-precision multigrid cycle, BiCGStab on the coarse grid, and a
Schwarz Alternating Procedure (SAP) smoother whose block systems are solved
by a fixed number of minimal-residual (MINRES) steps, with 16 or 24 null
space vectors.  It prints no algorithmic detail beyond that.  Readings taken
(the DD-alpha-AMG construction):

* blocks of ``block`` sites (each extent divides the lattice extent, the
  number of blocks per direction even); an aggregate is one block and one
  chirality (spins 0, 1 or 2, 3), so D^dag = g5 D g5 carries over to the
  coarse operator;
* the prolongation P maps coarse vector c[block][chirality][i] to
  sum_i c q_i, where q_i (i < Nv) is an orthonormal basis (by Gram-Schmidt
  in the order given) of the null vectors restricted to the aggregate;
  the restriction is P^dag;
* the coarse operator is D_c = P^dag D P;
* SAP: blocks coloured by the parity of their block coordinates; a cycle
  visits colour 0 then colour 1, each time recomputing the residual
  r = b - D x and adding to x, on every block of that colour, an
  approximate solution of D_B e = r_B, where D_B is D with every hop that
  leaves the block dropped, by a fixed number of minimal-residual steps
  from e = 0;
* the cycle M r: e_c = (approximate) solution of D_c e_c = P^dag r; z = P e_c;
  then z += SAP(r - D z) (post-smoothing only);
* FBiCGStab: BiCGStab with the preconditioner applied to the search
  directions (p^ = M p, s^ = M s), so M may change between applications;
* the coarse BiCGStab may run on the even-odd preconditioned coarse system
  (coarse sites split by the parity of their block coordinates, which every
  hopping coupling of D_c flips): with A the self couplings and H the
  hopping part, (1 - A_E^-1 H_EO A_O^-1 H_OE) e_E = A_E^-1 (r_E - H_EO
  A_O^-1 r_O) and e_O = A_O^-1 (r_O - H_OE e_E) (the paper names BiCGStab
  for the coarse grid and does not say whether it is preconditioned).

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""

from __future__ import annotations

import numpy as np

from . import dirac
from . import gamma as _g
from .lattice import Lattice
from .solvers import dot, norm


class Blocks:
    """Blocking of a lattice into SAP blocks / aggregates."""

    def __init__(self, lat: Lattice, block):
        self.lat, self.block = lat, tuple(int(b) for b in block)
        L = lat.dims
        if any(L[m] % self.block[m] for m in range(4)):
            raise ValueError("block extents must divide the lattice extents")
        self.cdims = tuple(L[m] // self.block[m] for m in range(4))
        if any(c % 2 for c in self.cdims):
            raise ValueError("the number of blocks per direction must be even")
        bc = [lat.coords[m] // self.block[m] for m in range(4)]
        cx, cy, cz, _ = self.cdims
        self.of_site = bc[0] + cx * (bc[1] + cy * (bc[2] + cz * bc[3]))
        self.nblocks = int(np.prod(self.cdims))
        bcoords = np.stack(np.unravel_index(np.arange(self.nblocks), self.cdims[::-1])[::-1])
        self.colour = bcoords.sum(axis=0) % 2
        self.sites = [np.nonzero(self.of_site == k)[0] for k in range(self.nblocks)]

    def inside(self, x, y) -> bool:
        return self.of_site[x] == self.of_site[y]


def block_dirac(U, psi, lat: Lattice, blocks: Blocks, kappa, csw, bc=(1, 1, 1, -1), T=None):
    """D_B psi for every block at once: D with every hop that leaves its block dropped."""
    if T is None:
        T = dirac.clover_term(U, lat, kappa, csw)
    x = np.arange(lat.V)
    out = dirac.apply_site(T, psi)
    for mu in range(4):
        g = _g.GAMMA[mu]
        j, wraps = lat.neighbor(x, mu, +1)
        keep = (blocks.of_site[j] == blocks.of_site[x]) * np.where(wraps, bc[mu], 1.0)
        chi = keep[:, None, None] * psi[j]
        out -= kappa * np.einsum("st,ntc->nsc", _g.I4 - g, chi @ np.swapaxes(U[mu], -1, -2))
        j, wraps = lat.neighbor(x, mu, -1)
        keep = (blocks.of_site[j] == blocks.of_site[x]) * np.where(wraps, bc[mu], 1.0)
        chi = keep[:, None, None] * psi[j]
        out -= kappa * np.einsum("st,ntc->nsc", _g.I4 + g, chi @ np.conj(U[mu][j]))
    return out


CHIRAL = (slice(0, 2), slice(2, 4))


class Multigrid:
    """The two-level construction for one gauge field, clover operator and null space."""

    def __init__(self, U, lat: Lattice, kappa, csw, block, null_vectors, bc=(1, 1, 1, -1)):
        self.U, self.lat, self.kappa, self.csw, self.bc = U, lat, kappa, csw, tuple(bc)
        self.blocks = Blocks(lat, block)
        self.T = dirac.clover_term(U, lat, kappa, csw)
        nv = np.asarray(null_vectors)
        self.nv = nv.shape[0]
        # Q[b][chi]: (len(block sites) * 6, Nv) orthonormal columns by Gram-Schmidt
        self.Q = []
        for b in range(self.blocks.nblocks):
            s = self.blocks.sites[b]
            qs = []
            for chi in range(2):
                A = nv[:, s][:, :, CHIRAL[chi], :].reshape(self.nv, -1).T.copy()
                for i in range(self.nv):
                    for j in range(i):
                        A[:, i] -= np.vdot(A[:, j], A[:, i]) * A[:, j]
                    A[:, i] /= np.linalg.norm(A[:, i])
                qs.append(A)
            self.Q.append(qs)

    # --- transfer -------------------------------------------------------------------
    def restrict(self, v):
        """P^dag v: shape (nblocks, 2, Nv)."""
        out = np.zeros((self.blocks.nblocks, 2, self.nv), dtype=np.complex128)
        for b in range(self.blocks.nblocks):
            s = self.blocks.sites[b]
            for chi in range(2):
                out[b, chi] = self.Q[b][chi].conj().T @ v[s][:, CHIRAL[chi], :].reshape(-1)
        return out

    def prolong(self, c):
        """P c: a fine spinor (V, 4, 3)."""
        out = np.zeros((self.lat.V, 4, 3), dtype=np.complex128)
        for b in range(self.blocks.nblocks):
            s = self.blocks.sites[b]
            for chi in range(2):
                out[s, CHIRAL[chi], :] = (self.Q[b][chi] @ c[b, chi]).reshape(len(s), 2, 3)
        return out

    # --- operators --------------------------------------------------------------------
    def D(self, psi):
        return dirac.dirac(self.U, psi, self.lat, self.kappa, self.csw, self.bc, T=self.T)

    def coarse_dense(self):
        """D_c = P^dag D P as a dense matrix over (block, chirality, vector), built column by column
        (once; cached)."""
        if getattr(self, "_Dc", None) is not None:
            return self._Dc
        n = self.blocks.nblocks * 2 * self.nv
        M = np.zeros((n, n), dtype=np.complex128)
        for k in range(n):
            e = np.zeros(n, dtype=np.complex128)
            e[k] = 1.0
            M[:, k] = self.restrict(self.D(self.prolong(e.reshape(-1, 2, self.nv)))).reshape(-1)
        self._Dc = M
        return M

    def coarse_evenodd_solve(self, rc, tol=1e-12, maxiter=5000):
        """D_c e = rc through the even-odd preconditioned coarse system (see the
        module docstring), BiCGStab on the even sites; built from the dense D_c."""
        from . import solvers

        Dc = self.coarse_dense()
        colour = np.repeat(self.blocks.colour, 2 * self.nv)
        E, O = colour == 0, colour == 1
        A_E, H_EO = Dc[np.ix_(E, E)], Dc[np.ix_(E, O)]
        H_OE, A_O = Dc[np.ix_(O, E)], Dc[np.ix_(O, O)]
        r = rc.reshape(-1)
        AOinv_rO = np.linalg.solve(A_O, r[O])
        rhs = np.linalg.solve(A_E, r[E] - H_EO @ AOinv_rO)

        def schur(v):
            return v - np.linalg.solve(A_E, H_EO @ np.linalg.solve(A_O, H_OE @ v))

        e_E, info = solvers.bicgstab(schur, rhs, tol=tol, maxiter=maxiter)
        e = np.zeros_like(r)
        e[E] = e_E
        e[O] = np.linalg.solve(A_O, r[O] - H_OE @ e_E)
        return e.reshape(rc.shape), info

    # --- SAP smoother -----------------------------------------------------------------
    def mr(self, rb, colour, steps):
        """`steps` minimal-residual steps on D_B e = r_B from e = 0, for every
        block of one colour at once (the blocks do not couple under D_B; each
        has its own step length alpha = <q, rho> / <q, q>, q = D_B rho)."""
        mask = (self.blocks.colour[self.blocks.of_site] == colour)[:, None, None]
        e = np.zeros_like(rb)
        rho = rb * mask
        for _ in range(steps):
            q = block_dirac(self.U, rho, self.lat, self.blocks, self.kappa, self.csw, self.bc, self.T) * mask
            for blk in np.nonzero(self.blocks.colour == colour)[0]:
                s = self.blocks.sites[blk]
                qq = np.vdot(q[s], q[s]).real
                alpha = np.vdot(q[s], rho[s]) / qq if qq > 0 else 0.0
                e[s] += alpha * rho[s]
                rho[s] -= alpha * q[s]
        return e

    def sap(self, b, cycles, mr_steps):
        """Approximate solution of D x = b by `cycles` SAP cycles from x = 0."""
        x = np.zeros_like(b)
        for _ in range(cycles):
            for colour in (0, 1):
                x = x + self.mr(b - self.D(x), colour, mr_steps)
        return x

    # --- the cycle and the outer solver ----------------------------------------------
    def cycle(self, r, cycles=2, mr_steps=4, coarse_solve=None):
        """M r: coarse correction, then SAP post-smoothing on the remaining residual."""
        rc = self.restrict(r)
        if coarse_solve is None:
            ec = np.linalg.solve(self.coarse_dense(), rc.reshape(-1)).reshape(rc.shape)
        else:
            ec = coarse_solve(rc)
        z = self.prolong(ec)
        return z + self.sap(r - self.D(z), cycles, mr_steps)


def fbicgstab(A, M, b, tol=1e-12, maxiter=1000):
    """Flexible BiCGStab: BiCGStab for A x = b with the search directions
    preconditioned, p^ = M(p), s^ = M(s) (M may vary between calls)."""
    bnorm = norm(b)
    x = np.zeros_like(b)
    info = {"iters": 0, "converged": False, "true_rel_residual": 0.0}
    if bnorm == 0.0:
        info["converged"] = True
        return x, info
    r = b.copy()
    rhat = r.copy()
    rho = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    while info["iters"] < maxiter and norm(r) > tol * bnorm:
        rho_new = dot(rhat, r)
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = M(p)
        v = A(ph)
        alpha = rho_new / dot(rhat, v)
        s = r - alpha * v
        sh = M(s)
        t = A(sh)
        tt = dot(t, t).real
        omega = dot(t, s) / tt if tt > 0 else 0.0
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_new
        info["iters"] += 1
    info["true_rel_residual"] = norm(b - A(x)) / bnorm
    info["converged"] = info["true_rel_residual"] <= tol * 10
    return x, info
