"""Checks that pin the oracle to mathematics other than itself.

Each function returns an error measure; tests/test_oracle_pins.py asserts it
is at rounding level for the oracle as written, and tests/test_oracle_mutations.py
asserts it is large once a plausible mistake is planted in the oracle.
"""

from __future__ import annotations

import numpy as np

import synth
from oracle import dirac, domainwall, evenodd, gamma, multigrid, solvers, staggered
from oracle.lattice import Lattice


def rel(a, b) -> float:
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    n = np.linalg.norm(np.asarray(b))
    return float(d / n) if n > 0 else float(d)


# --- free field: plane waves are eigenvectors of D_W with a closed-form eigenvalue ---


def plane_wave(lat: Lattice, n, u):
    """psi(x) = exp(i p.x) u with p_k = 2 pi n_k / L_k and p_t = (2 n_t + 1) pi / L_t."""
    L = lat.dims
    p = [2 * np.pi * n[k] / L[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / L[3]]
    phase = np.exp(1j * sum(p[mu] * lat.coords[mu] for mu in range(4)))
    return phase[:, None, None] * u[None], p


def free_field_symbol(p, kappa):
    """The closed form D_W(p) = 1 - 2 kappa sum cos p_mu + 2 i kappa sum gamma_mu sin p_mu."""
    M = (1 - 2 * kappa * sum(np.cos(q) for q in p)) * np.eye(4, dtype=np.complex128)
    for mu in range(4):
        M = M + 2j * kappa * np.sin(p[mu]) * PINNED_GAMMA[mu]
    return M


def _pinned_gamma():
    """The chiral basis, typed here independently of oracle.gamma."""
    s = [np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]])]
    z = np.zeros((2, 2))
    e = np.eye(2)
    g = [np.block([[z, -1j * s[k]], [1j * s[k], z]]) for k in range(3)]
    g.append(np.block([[z, e], [e, z]]))
    return [x.astype(np.complex128) for x in g]


PINNED_GAMMA = _pinned_gamma()


def free_field_error(dims=(4, 6, 4, 8), kappa=0.12, modes=((0, 0, 0, 0), (1, 2, 3, 1), (3, 5, 1, 6)), seed=7):
    lat = Lattice(dims)
    U = synth.unit_gauge(dims)
    gen = np.random.default_rng(seed)
    err = 0.0
    for n in modes:
        u = gen.standard_normal((4, 3)) + 1j * gen.standard_normal((4, 3))
        psi, p = plane_wave(lat, n, u)
        got = dirac.wilson(U, psi, lat, kappa)
        want = np.einsum("st,ntc->nsc", free_field_symbol(p, kappa), psi)
        err = max(err, rel(got, want))
    return err


def free_field_inverse_error(dims=(4, 4, 4, 8), kappa=0.12, n=(1, 0, 2, 3), seed=3):
    """BiCGStab on D_W applied to a plane wave reproduces the closed-form inverse."""
    lat = Lattice(dims)
    U = synth.unit_gauge(dims)
    gen = np.random.default_rng(seed)
    u = gen.standard_normal((4, 3)) + 1j * gen.standard_normal((4, 3))
    b, p = plane_wave(lat, n, u)
    x, info = solvers.bicgstab(lambda v: dirac.wilson(U, v, lat, kappa), b, tol=1e-13)
    Minv = np.linalg.inv(free_field_symbol(p, kappa))
    want = np.einsum("st,ntc->nsc", Minv, b)
    return rel(x, want)


# --- gamma_5 hermiticity -----------------------------------------------------------


def gamma5_hermiticity_error(dims=(4, 4, 6, 4), kappa=0.13, csw=1.3, eps=0.4, seed=11):
    """<phi, g5 D g5 psi> = <D phi, psi> for random fields."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    phi = synth.gaussian_spinor(dims, seed, field_id=5)
    psi = synth.gaussian_spinor(dims, seed, field_id=6)
    g5 = np.diag([1, 1, -1, -1]).astype(np.complex128)
    g5v = lambda v: np.einsum("st,ntc->nsc", g5, v)  # noqa: E731
    lhs = np.vdot(phi, g5v(dirac.dirac(U, g5v(psi), lat, kappa, csw)))
    rhs = np.vdot(dirac.dirac(U, phi, lat, kappa, csw), psi)
    return abs(lhs - rhs) / (np.linalg.norm(phi) * np.linalg.norm(psi))


# --- gauge covariance --------------------------------------------------------------


def random_su3(n, gen):
    z = gen.standard_normal((n, 3, 3)) + 1j * gen.standard_normal((n, 3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(q)
    return q / (det ** (1 / 3))[:, None, None]


def gauge_transform(U, lat: Lattice, Om):
    """U_mu(x) -> Om(x) U_mu(x) Om(x + mu)^dagger."""
    out = np.empty_like(U)
    x = np.arange(lat.V)
    for mu in range(4):
        y, _ = lat.neighbor(x, mu, +1)
        out[mu] = Om @ U[mu] @ np.conj(np.swapaxes(Om[y], -1, -2))
    return out


def covariance_error(dims=(4, 6, 4, 4), kappa=0.12, csw=1.1, eps=0.5, seed=21):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    gen = np.random.default_rng(seed)
    Om = random_su3(lat.V, gen)
    Ug = gauge_transform(U, lat, Om)
    psi = synth.gaussian_spinor(dims, seed, field_id=4)
    rot = lambda v: np.einsum("nab,nsb->nsa", Om, v)  # noqa: E731
    lhs = dirac.dirac(Ug, rot(psi), lat, kappa, csw)
    rhs = rot(dirac.dirac(U, psi, lat, kappa, csw))
    return rel(lhs, rhs)


# --- abelian flux: F_{mu nu} known exactly ----------------------------------------


def abelian_flux_links(lat: Lattice, mu, nu, n_flux, a, b):
    """U_mu = exp(-i phi x_nu D), U_nu = exp(i phi L_nu x_mu D) on the last nu slice.

    Every plaquette in the (mu, nu) plane then equals exp(i phi D) with
    phi = 2 pi n / (L_mu L_nu) and D = diag(a, b, -a-b); all other planes are flat.
    """
    L = lat.dims
    phi = 2 * np.pi * n_flux / (L[mu] * L[nu])
    D = np.array([a, b, -a - b], dtype=float)
    U = synth.unit_gauge(lat.dims)
    xm, xn = lat.coords[mu], lat.coords[nu]
    U[mu] = np.einsum("nk,kl->nkl", np.exp(-1j * phi * xn[:, None] * D[None]), np.eye(3))
    last = xn == L[nu] - 1
    ph = np.where(last[:, None], np.exp(1j * phi * L[nu] * xm[:, None] * D[None]), 1.0)
    U[nu] = np.einsum("nk,kl->nkl", ph, np.eye(3))
    return U, phi, D


def abelian_flux_error(dims=(4, 6, 4, 8), kappa=0.11, csw=1.7):
    """F and T from the oracle against sin(phi D) minus its trace, in every plane."""
    lat = Lattice(dims)
    err = 0.0
    x = np.arange(lat.V)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            U, phi, D = abelian_flux_links(lat, mu, nu, 1, 1, 2)
            f = np.sin(phi * D)
            f = f - f.sum() / 3
            for r in range(4):
                for s in range(r + 1, 4):
                    F = dirac.field_strength(U, lat, x, r, s)
                    want = np.diag(f) if (r, s) == (mu, nu) else np.zeros((3, 3))
                    err = max(err, float(np.max(np.abs(F - want[None]))))
            T = dirac.clover_term(U, lat, kappa, csw, x)
            sig = 0.5j * (PINNED_GAMMA[mu] @ PINNED_GAMMA[nu] - PINNED_GAMMA[nu] @ PINNED_GAMMA[mu])
            Twant = np.eye(12) - kappa * csw * np.kron(sig, np.diag(f))
            err = max(err, float(np.max(np.abs(T - Twant[None]))))
    return err


# --- even-odd algebra (Eq. 1) -----------------------------------------------------


def schur_dense_error(dims=(2, 2, 2, 2), kappa=0.12, csw=1.0, eps=0.6, seed=31):
    """D^(eo) from the blocks equals T_ee^-1 (T_ee - D_eo T_oo^-1 D_oe) from the dense matrix."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    M = solvers.dense_dirac(U, lat, kappa, csw)
    e = np.concatenate([np.arange(12 * s, 12 * s + 12) for s in lat.even])
    o = np.concatenate([np.arange(12 * s, 12 * s + 12) for s in lat.odd])
    Mee, Meo, Moe, Moo = M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)]
    S = np.linalg.solve(Mee, Mee - Meo @ np.linalg.solve(Moo, Moe))
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    n = 12 * len(lat.even)
    Sb = solvers.dense_matrix(lambda v: eo.schur(v.reshape(-1, 4, 3)).reshape(-1), n)
    return rel(Sb, S)


def dense_vs_stencil_error(dims=(2, 2, 2, 4), kappa=0.13, csw=0.9, eps=0.5, seed=41):
    """The stencil D equals the matrix filled from its matrix elements."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    M = solvers.dense_dirac(U, lat, kappa, csw)
    Mb = solvers.dense_matrix(lambda v: dirac.dirac(U, v.reshape(-1, 4, 3), lat, kappa, csw).reshape(-1), 12 * lat.V)
    return rel(Mb, M)


def lu_vs_bicgstab_error(dims=(2, 2, 2, 2), kappa=0.12, csw=1.0, eps=0.5, seed=51, evenodd_solve=False, maxiter=100000):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    b = synth.gaussian_spinor(dims, seed)
    M = solvers.dense_dirac(U, lat, kappa, csw)
    x_lu = solvers.lu_solve(M, b.reshape(-1)).reshape(b.shape)
    if evenodd_solve:
        eo = evenodd.EvenOdd(U, lat, kappa, csw)
        xe, info = solvers.bicgstab(eo.schur, eo.prepare(b), tol=1e-14, maxiter=maxiter)
        x = eo.reconstruct(xe, b)
    else:
        x, info = solvers.bicgstab(lambda v: dirac.dirac(U, v, lat, kappa, csw), b, tol=1e-14, maxiter=maxiter)
    return rel(x, x_lu)


def evenodd_vs_full_error(dims=(4, 4, 4, 4), kappa=0.12, csw=1.0, eps=0.3, seed=61):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    b = synth.gaussian_spinor(dims, seed)
    T = dirac.clover_term(U, lat, kappa, csw)
    x_full, _ = solvers.bicgstab(lambda v: dirac.dirac(U, v, lat, kappa, csw, T=T), b, tol=1e-13)
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    xe, _ = solvers.bicgstab(eo.schur, eo.prepare(b), tol=1e-13)
    x_eo = eo.reconstruct(xe, b)
    return rel(x_eo, x_full)


def blocks_vs_full_error(dims=(4, 2, 6, 4), kappa=0.12, csw=1.2, eps=0.4, seed=71):
    """The 2x2 block form of Eq. 1 reassembles the full operator."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    psi = synth.gaussian_spinor(dims, seed)
    eo = evenodd.EvenOdd(U, lat, kappa, csw)
    return rel(eo.full(psi), dirac.dirac(U, psi, lat, kappa, csw))


def gamma_algebra_error():
    err = 0.0
    G = gamma.GAMMA
    for mu in range(4):
        err = max(err, np.abs(G[mu] - G[mu].conj().T).max())
        for nu in range(4):
            anti = G[mu] @ G[nu] + G[nu] @ G[mu]
            err = max(err, np.abs(anti - 2 * (mu == nu) * np.eye(4)).max())
    err = max(err, np.abs(gamma.gamma5() - np.diag([1, 1, -1, -1])).max())
    for mu in range(4):
        err = max(err, np.abs(G[mu] - PINNED_GAMMA[mu]).max())
    return float(err)


# --- Moebius domain wall -------------------------------------------------------------
#
# Closed form used below (the overlap relation of domain-wall fermions): with
# K = (b + c) W (2 + (b - c) W)^-1 and the polar approximation
#     eps_Ls(h) = ((1 + h)^Ls - (1 - h)^Ls) / ((1 + h)^Ls + (1 - h)^Ls)
# of the sign function applied to the Hermitian gamma_5 K, the four-dimensional
# operator seen by the boundary fields q = P_- psi_0 + P_+ psi_{Ls-1} is
#     D_eff(m_f) = (1 + m_f)/2 + (1 - m_f)/2 gamma_5 eps_Ls(gamma_5 K),
# and it is reached from the five-dimensional operator as
#     D_eff(m_f) chi = q( D(1)^-1 D(m_f) psi_chi ),  psi_chi = P_- chi at s = 0, P_+ chi at s = Ls-1.


def _eps_polar(Hm, Ls):
    lam, Q = np.linalg.eigh(Hm)
    e = ((1 + lam) ** Ls - (1 - lam) ** Ls) / ((1 + lam) ** Ls + (1 - lam) ** Ls)
    return (Q * e) @ Q.conj().T


def _deff_closed_form(W, b, c, mf, Ls, g5):
    n = W.shape[0]
    K = np.linalg.solve(2 * np.eye(n) + (b - c) * W, (b + c) * W)
    return (1 + mf) / 2 * np.eye(n) + (1 - mf) / 2 * g5 @ _eps_polar(g5 @ K, Ls)


def _deff_from_5d(op1, opm, chis):
    """D_eff chi for each chi in chis via the five-dimensional operators (dense LU for D(1))."""
    Ls, V = op1.Ls, op1.lat.V
    n5 = Ls * V * 12
    D1 = solvers.dense_matrix(lambda v: op1.full(v.reshape(Ls, V, 4, 3)).reshape(-1), n5)
    out = []
    for chi in chis:
        psi = np.zeros((Ls, V, 4, 3), dtype=np.complex128)
        psi[0][:, 2:] = chi[:, 2:]
        psi[Ls - 1][:, :2] = chi[:, :2]
        z = np.linalg.solve(D1, opm.full(psi).reshape(-1)).reshape(Ls, V, 4, 3)
        q = np.zeros_like(chi)
        q[:, 2:] = z[0][:, 2:]
        q[:, :2] = z[Ls - 1][:, :2]
        out.append(q)
    return out


def mobius_overlap_error(dims=(2, 2, 2, 2), Ls=4, M5=1.8, b=1.5, c=0.5, mf=0.07, eps=0.5, seed=81):
    """The oracle's 5-d Moebius operator reproduces the overlap closed form on a random gauge field.

    W = D_W(-M5) comes from the dense Wilson matrix filled from its matrix
    elements (solvers.dense_dirac, pinned on its own): with kappa = 1 that
    matrix is 1 - H.
    """
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    n4 = 12 * lat.V
    H = np.eye(n4) - solvers.dense_dirac(U, lat, 1.0, 0.0)
    W = (4.0 - M5) * np.eye(n4) - 0.5 * H
    g5 = np.kron(np.eye(lat.V), np.kron(np.diag([1.0, 1.0, -1.0, -1.0]), np.eye(3)))
    want = _deff_closed_form(W, b, c, mf, Ls, g5)
    gen = np.random.default_rng(seed)
    chis = [gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3)) for _ in range(3)]
    got = _deff_from_5d(domainwall.Mobius(U, lat, Ls, M5, b, c, 1.0), domainwall.Mobius(U, lat, Ls, M5, b, c, mf), chis)
    return max(rel(g.reshape(-1), want @ chi.reshape(-1)) for g, chi in zip(got, chis))


def mobius_free_field_error(dims=(4, 2, 2, 2), Ls=4, M5=1.8, b=1.5, c=0.5, mf=0.05,
                            modes=((0, 0, 0, 0), (1, 0, 1, 0), (3, 1, 0, 1)), seed=83):
    """Free field: plane waves give the overlap closed form with the Fourier symbol
    W(p) = (4 - M5) - sum cos p_mu + i sum gamma_mu sin p_mu (a 4x4 spin matrix)."""
    lat = Lattice(dims)
    U = synth.unit_gauge(dims)
    gen = np.random.default_rng(seed)
    g5 = np.diag([1.0, 1.0, -1.0, -1.0]).astype(np.complex128)
    chis, wants = [], []
    for n in modes:
        u = gen.standard_normal((4, 3)) + 1j * gen.standard_normal((4, 3))
        chi, p = plane_wave(lat, n, u)
        Wp = (4.0 - M5 - sum(np.cos(q) for q in p)) * np.eye(4, dtype=np.complex128)
        for mu in range(4):
            Wp = Wp + 1j * np.sin(p[mu]) * PINNED_GAMMA[mu]
        Dp = _deff_closed_form(Wp, b, c, mf, Ls, g5)
        chis.append(chi)
        wants.append(np.einsum("st,ntc->nsc", Dp, chi))
    got = _deff_from_5d(domainwall.Mobius(U, lat, Ls, M5, b, c, 1.0), domainwall.Mobius(U, lat, Ls, M5, b, c, mf), chis)
    return max(rel(g, w) for g, w in zip(got, wants))


def _mobius(dims, Ls, eps, seed, M5=1.8, b=1.5, c=0.5, mf=0.1):
    lat = Lattice(dims)
    return domainwall.Mobius(synth.gauge_field(dims, eps, seed), lat, Ls, M5, b, c, mf)


def mobius_schur_dense_error(dims=(2, 2, 2, 2), Ls=3, eps=0.5, seed=85):
    """D^(eo) and the even-odd solve against the dense 5-d matrix: the Schur
    complement A_ee^-1 (A_ee - D_eo A_oo^-1 D_oe) of its parity blocks, and LU."""
    op = _mobius(dims, Ls, eps, seed)
    lat, V = op.lat, op.lat.V
    M = solvers.dense_matrix(lambda v: op.full(v.reshape(Ls, V, 4, 3)).reshape(-1), Ls * V * 12)
    idx = np.arange(Ls * V * 12).reshape(Ls, V, 12)
    e, o = idx[:, lat.even].reshape(-1), idx[:, lat.odd].reshape(-1)
    Mee, Meo, Moe, Moo = M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)]
    S = np.linalg.solve(Mee, Mee - Meo @ np.linalg.solve(Moo, Moe))
    ne = len(e)
    Sb = solvers.dense_matrix(lambda v: op.schur(v.reshape(Ls, -1, 4, 3)).reshape(-1), ne)
    err = rel(Sb, S)
    rhs = synth.gaussian_spinor(dims, seed, nrhs=Ls)
    x_lu = np.linalg.solve(M, rhs.reshape(-1)).reshape(rhs.shape)
    xe = np.linalg.solve(Sb, op.prepare(rhs).reshape(-1)).reshape(Ls, -1, 4, 3)
    return max(err, rel(op.reconstruct(xe, rhs), x_lu))


def mobius_adjoint_error(dims=(4, 2, 2, 4), Ls=5, eps=0.5, seed=87):
    """<u, D^(eo) v> = <D^(eo)^dagger u, v> for random u, v."""
    op = _mobius(dims, Ls, eps, seed)
    vh = op.lat.V // 2
    gen = np.random.default_rng(seed)
    u = gen.standard_normal((Ls, vh, 4, 3)) + 1j * gen.standard_normal((Ls, vh, 4, 3))
    v = gen.standard_normal((Ls, vh, 4, 3)) + 1j * gen.standard_normal((Ls, vh, 4, 3))
    lhs, rhs = np.vdot(u, op.schur(v)), np.vdot(op.schur_dag(u), v)
    return abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(op.schur(v)))


def shamir_reflection_error(dims=(2, 2, 4, 2), Ls=4, eps=0.5, seed=89):
    """Shamir (b = 1, c = 0): gamma_5 R_5 D gamma_5 R_5 = D^dagger, R_5: s -> Ls-1-s."""
    op = _mobius(dims, Ls, eps, seed, b=1.0, c=0.0)
    gen = np.random.default_rng(seed)
    sh = (Ls, op.lat.V, 4, 3)
    u = gen.standard_normal(sh) + 1j * gen.standard_normal(sh)
    v = gen.standard_normal(sh) + 1j * gen.standard_normal(sh)
    g5r5 = lambda w: (w[::-1] * np.array([1, 1, -1, -1])[None, None, :, None])  # noqa: E731
    lhs = np.vdot(u, g5r5(op.full(g5r5(v))))
    rhs = np.vdot(op.full(u), v)
    return abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(v))


def cg_error(n=48, seed=91, maxiter=400):
    """CG on a random Hermitian positive definite matrix against LAPACK, and
    CG on the normal equations of the even-odd Moebius system against LU."""
    gen = np.random.default_rng(seed)
    Z = gen.standard_normal((n, n)) + 1j * gen.standard_normal((n, n))
    A = Z @ Z.conj().T + 0.5 * np.eye(n)
    b = gen.standard_normal(n) + 1j * gen.standard_normal(n)
    x, _ = solvers.cg(lambda v: A @ v, b, tol=1e-13, maxiter=maxiter)
    err = rel(x, np.linalg.solve(A, b))
    op = _mobius((2, 2, 2, 2), 3, 0.5, seed)
    ne = 3 * op.lat.V // 2 * 12
    S = solvers.dense_matrix(lambda v: op.schur(v.reshape(3, -1, 4, 3)).reshape(-1), ne)
    bh = gen.standard_normal((3, op.lat.V // 2, 4, 3)) + 1j * gen.standard_normal((3, op.lat.V // 2, 4, 3))
    xe, _ = solvers.cgnr(op.schur, op.schur_dag, bh, tol=1e-13, maxiter=maxiter)
    return max(err, rel(xe.reshape(-1), np.linalg.solve(S, bh.reshape(-1))))


# --- staggered --------------------------------------------------------------------------


def staggered_free_field_error(dims=(4, 6, 4, 8), mass=0.05, modes=((0, 0, 0, 0), (1, 2, 3, 1), (3, 5, 1, 6)), seed=101):
    """Free field: D^dagger D = m^2 + sum_mu sin^2 p_mu on plane waves, with
    D^dagger = 2m - D (the hopping term is anti-Hermitian)."""
    lat = Lattice(dims)
    U = synth.unit_gauge(dims)
    op = staggered.Staggered(U, lat, mass)
    gen = np.random.default_rng(seed)
    L = lat.dims
    err = 0.0
    for n in modes:
        p = [2 * np.pi * n[k] / L[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / L[3]]
        phase = np.exp(1j * sum(p[mu] * lat.coords[mu] for mu in range(4)))
        u = gen.standard_normal(3) + 1j * gen.standard_normal(3)
        chi = phase[:, None] * u[None]
        Dchi = op.full(chi)
        DdD = 2 * mass * Dchi - op.full(Dchi)
        want = (mass**2 + sum(np.sin(q) ** 2 for q in p)) * chi
        err = max(err, rel(DdD, want))
    return err


def staggered_antihermitian_error(dims=(4, 4, 6, 4), eps=0.5, seed=103):
    """<u, H v> = -<H u, v> for the hopping term on a random gauge field."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    gen = np.random.default_rng(seed)
    u = gen.standard_normal((lat.V, 3)) + 1j * gen.standard_normal((lat.V, 3))
    v = gen.standard_normal((lat.V, 3)) + 1j * gen.standard_normal((lat.V, 3))
    lhs = np.vdot(u, staggered.hop(U, v, lat))
    rhs = -np.vdot(staggered.hop(U, u, lat), v)
    return abs(lhs - rhs) / (np.linalg.norm(u) * np.linalg.norm(v))


def staggered_covariance_error(dims=(4, 6, 4, 4), mass=0.1, eps=0.5, seed=105):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    gen = np.random.default_rng(seed)
    Om = random_su3(lat.V, gen)
    Ug = gauge_transform(U, lat, Om)
    chi = gen.standard_normal((lat.V, 3)) + 1j * gen.standard_normal((lat.V, 3))
    rot = lambda v: np.einsum("nab,nb->na", Om, v)  # noqa: E731
    return rel(staggered.Staggered(Ug, lat, mass).full(rot(chi)), rot(staggered.Staggered(U, lat, mass).full(chi)))


def dense_staggered(U, lat: Lattice, mass: float, bc=(1, 1, 1, -1)) -> np.ndarray:
    """D as a dense (3V x 3V) matrix filled from its matrix elements with explicit loops:
    m on the diagonal, +eta bc U_mu(x)/2 at y = x + mu, -eta bc U_mu(x - mu)^dag / 2 at y = x - mu."""
    V = lat.V
    M = np.zeros((3 * V, 3 * V), dtype=np.complex128)
    for x in range(V):
        M[3 * x : 3 * x + 3, 3 * x : 3 * x + 3] += mass * np.eye(3)
        c = lat.coords[:, x]
        for mu in range(4):
            e = (-1.0) ** int(sum(c[:mu]))
            (y,), (w,) = lat.neighbor(np.array([x]), mu, +1)
            ph = bc[mu] if w else 1.0
            M[3 * x : 3 * x + 3, 3 * y : 3 * y + 3] += 0.5 * e * ph * U[mu][x]
            (y,), (w,) = lat.neighbor(np.array([x]), mu, -1)
            ph = bc[mu] if w else 1.0
            M[3 * x : 3 * x + 3, 3 * y : 3 * y + 3] -= 0.5 * e * ph * U[mu][y].conj().T
    return M


def staggered_dense_error(dims=(2, 2, 2, 4), mass=0.1, eps=0.5, seed=107):
    """The stencil against the dense matrix; the Schur operator against the dense
    Schur complement; the even-odd CG solve against LU."""
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    op = staggered.Staggered(U, lat, mass)
    M = dense_staggered(U, lat, mass)
    Mb = solvers.dense_matrix(lambda v: op.full(v.reshape(-1, 3)).reshape(-1), 3 * lat.V)
    err = rel(Mb, M)
    e = np.concatenate([np.arange(3 * s, 3 * s + 3) for s in lat.even])
    o = np.concatenate([np.arange(3 * s, 3 * s + 3) for s in lat.odd])
    Mee, Meo, Moe, Moo = M[np.ix_(e, e)], M[np.ix_(e, o)], M[np.ix_(o, e)], M[np.ix_(o, o)]
    S = np.linalg.solve(Mee, Mee - Meo @ np.linalg.solve(Moo, Moe))
    Sb = solvers.dense_matrix(lambda v: op.schur(v.reshape(-1, 3)).reshape(-1), len(e))
    err = max(err, rel(Sb, S))
    gen = np.random.default_rng(seed)
    b = gen.standard_normal((lat.V, 3)) + 1j * gen.standard_normal((lat.V, 3))
    x_lu = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    xe, _ = solvers.cg(op.normal_even, op.prepare(b), tol=1e-14, maxiter=2000)
    return max(err, rel(op.reconstruct(xe, b), x_lu))


# --- two-level multigrid -------------------------------------------------------------------


def _mg_case(dims=(4, 4, 4, 4), block=(2, 2, 2, 2), nv=3, kappa=0.12, csw=1.0, eps=0.4, seed=111):
    lat = Lattice(dims)
    U = synth.gauge_field(dims, eps, seed)
    gen = np.random.default_rng(seed)
    vs = gen.standard_normal((nv, lat.V, 4, 3)) + 1j * gen.standard_normal((nv, lat.V, 4, 3))
    return lat, U, multigrid.Multigrid(U, lat, kappa, csw, block, vs)


def _dense_P(mg):
    """P as a dense (12V x 2 Nb Nv) matrix assembled from the aggregate bases."""
    lat, nb, nv = mg.lat, mg.blocks.nblocks, mg.nv
    P = np.zeros((12 * lat.V, nb * 2 * nv), dtype=np.complex128)
    for b in range(nb):
        s = mg.blocks.sites[b]
        for chi in range(2):
            rows = np.array([12 * x + 6 * chi + k for x in s for k in range(6)])
            P[rows, (b * 2 + chi) * nv : (b * 2 + chi + 1) * nv] = mg.Q[b][chi]
    return P


def mg_transfer_error():
    """P^dag P = 1; restrict / prolong agree with the dense P; the aggregate
    bases span the null vectors restricted to each aggregate."""
    lat, U, mg = _mg_case()
    P = _dense_P(mg)
    err = np.abs(P.conj().T @ P - np.eye(P.shape[1])).max()
    gen = np.random.default_rng(5)
    c = gen.standard_normal((mg.blocks.nblocks, 2, mg.nv)) + 1j * gen.standard_normal((mg.blocks.nblocks, 2, mg.nv))
    err = max(err, rel(mg.prolong(c).reshape(-1), P @ c.reshape(-1)))
    v = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    err = max(err, rel(mg.restrict(v).reshape(-1), P.conj().T @ v.reshape(-1)))
    return float(err)


def mg_coarse_error():
    """D_c from the oracle equals P^dag M P with M the dense matrix-element form of D,
    and satisfies D_c^dag = G5 D_c G5 (G5 = +1 / -1 on the two chiral aggregates)."""
    lat, U, mg = _mg_case()
    P = _dense_P(mg)
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    Dc = mg.coarse_dense()
    err = rel(Dc, P.conj().T @ M @ P)
    g5 = np.tile(np.repeat([1.0, -1.0], mg.nv), mg.blocks.nblocks)
    err = max(err, rel(Dc.conj().T, g5[:, None] * Dc * g5[None, :]))
    return err


def mg_block_operator_error():
    """D_B equals the dense matrix with every entry between different blocks removed."""
    lat, U, mg = _mg_case(dims=(4, 2, 2, 2), block=(2, 1, 1, 1))
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    same = np.repeat(mg.blocks.of_site, 12)
    MB = M * (same[:, None] == same[None, :])
    f = lambda v: multigrid.block_dirac(U, v.reshape(-1, 4, 3), lat, mg.blocks, mg.kappa, mg.csw, T=mg.T).reshape(-1)  # noqa: E731
    return rel(solvers.dense_matrix(f, 12 * lat.V), MB)


def mg_sap_error():
    """With converged block solves, one SAP cycle is the two block-Gauss-Seidel
    half-sweeps written with dense block inverses; one MR step is the
    least-squares step on each block."""
    lat, U, mg = _mg_case(kappa=0.1)
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    site_block = np.repeat(mg.blocks.of_site, 12)
    gen = np.random.default_rng(9)
    b = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    bf = b.reshape(-1)
    x = np.zeros_like(bf)
    for colour in (0, 1):
        r = bf - M @ x
        for blk in np.nonzero(mg.blocks.colour == colour)[0]:
            idx = np.nonzero(site_block == blk)[0]
            x[idx] += np.linalg.solve(M[np.ix_(idx, idx)], r[idx])
    err = rel(mg.sap(b, 1, 200).reshape(-1), x)
    # one MR step on each colour-0 block against numpy's least squares
    e = mg.mr(b, 0, 1).reshape(-1)
    for blk in np.nonzero(mg.blocks.colour == 0)[0]:
        idx = np.nonzero(site_block == blk)[0]
        q = M[np.ix_(idx, idx)] @ bf[idx]
        a = np.linalg.lstsq(q[:, None], bf[idx], rcond=None)[0][0]
        err = max(err, rel(e[idx], a * bf[idx]))
    return err


def mg_cycle_error():
    """The cycle composed from dense pieces: z = P (P^dag M P)^-1 P^dag r, then one
    SAP cycle with converged block solves on r - M z."""
    lat, U, mg = _mg_case(kappa=0.1)
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    P = _dense_P(mg)
    site_block = np.repeat(mg.blocks.of_site, 12)
    gen = np.random.default_rng(17)
    r = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    rf = r.reshape(-1)
    z = P @ np.linalg.solve(P.conj().T @ M @ P, P.conj().T @ rf)
    b2 = rf - M @ z
    x = np.zeros_like(rf)
    for colour in (0, 1):
        res = b2 - M @ x
        for blk in np.nonzero(mg.blocks.colour == colour)[0]:
            idx = np.nonzero(site_block == blk)[0]
            x[idx] += np.linalg.solve(M[np.ix_(idx, idx)], res[idx])
    return rel(mg.cycle(r, 1, 200).reshape(-1), z + x)


def mg_solve_error():
    """FBiCGStab preconditioned by the two-level cycle (exact coarse solve)
    reaches the LU solution; with M = 1 it takes the BiCGStab iterates."""
    lat, U, mg = _mg_case(nv=4, kappa=0.124)
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    gen = np.random.default_rng(13)
    b = gen.standard_normal((lat.V, 4, 3)) + 1j * gen.standard_normal((lat.V, 4, 3))
    x_lu = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    x, info = multigrid.fbicgstab(mg.D, lambda r: mg.cycle(r, 2, 4), b, tol=1e-12, maxiter=200)
    err = rel(x, x_lu)
    x1, i1 = multigrid.fbicgstab(mg.D, lambda r: r, b, tol=1e-12, maxiter=500)
    x2, i2 = solvers.bicgstab(mg.D, b, tol=1e-12, maxiter=500)
    return max(err, rel(x1, x_lu), float(abs(i1["iters"] - i2["iters"]) > 1))


def mg_coarse_evenodd_error():
    """Every hopping coupling of D_c joins coarse sites of opposite colour (the
    same-colour blocks of the dense P^dag M P hold only the self couplings), and
    the even-odd coarse solve reaches the LU solution of the full coarse system."""
    lat, U, mg = _mg_case(nv=3, kappa=0.12)
    P = _dense_P(mg)
    M = solvers.dense_dirac(U, lat, mg.kappa, mg.csw)
    Dc = P.conj().T @ M @ P
    n2 = 2 * mg.nv
    colour = np.repeat(mg.blocks.colour, n2)
    site = np.repeat(np.arange(mg.blocks.nblocks), n2)
    same_colour_other_site = (colour[:, None] == colour[None, :]) & (site[:, None] != site[None, :])
    err = float(np.abs(Dc[same_colour_other_site]).max() / np.abs(Dc).max())
    gen = np.random.default_rng(23)
    rc = gen.standard_normal((mg.blocks.nblocks, 2, mg.nv)) + 1j * gen.standard_normal((mg.blocks.nblocks, 2, mg.nv))
    e, info = mg.coarse_evenodd_solve(rc, tol=1e-13)
    return max(err, rel(e.reshape(-1), np.linalg.solve(Dc, rc.reshape(-1))))

