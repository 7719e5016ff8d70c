"""Planted mistakes in the oracle must fail a pin.

Each case edits one line of the oracle's own source (a sign, a dropped term,
a transposed operand, a wrong index), loads the edited module, swaps its
functions in for the originals and checks that the named pin now reports a
large error.  This shows the pins in tests/pins.py can tell a wrong oracle
from a right one; nothing here touches a GPU.
"""

import importlib
import inspect

import pytest

import oracle
from tests import pins

MUTANTS = [
    # (module, original text, planted text, pin, threshold above every tolerance the pins use)
    ("dirac", "_spin(_g.I4 - g,", "_spin(_g.I4 + g,", pins.free_field_error, 1e-10),
    ("dirac", "_colour(_dag(U[mu][j]), phase * psi[j])", "_colour(U[mu][j], phase * psi[j])", pins.covariance_error, 1e-10),
    ("dirac", "phase = np.where(wraps, bc[mu], 1.0)[:, None, None]\n        out += _spin(_g.I4 - g",
     "phase = 1.0\n        out += _spin(_g.I4 - g", pins.free_field_error, 1e-10),
    ("dirac", "_colour(U[mu][sites], phase * psi[j])", "_colour(np.swapaxes(U[mu][sites], -1, -2), phase * psi[j])",
     pins.covariance_error, 1e-10),
    ("dirac", "j, wraps = lat.neighbor(sites, mu, -1)", "j, wraps = lat.neighbor(sites, mu, +1)", pins.free_field_error, 1e-10),
    ("dirac", "F = (Q - _dag(Q)) / 8j", "F = (Q - _dag(Q)) / 4j", pins.abelian_flux_error, 1e-10),
    ("dirac", "return F - (tr / 3.0)[:, None, None] * np.eye(3)", "return F", pins.abelian_flux_error, 1e-10),
    ("dirac", "q = q + Un[x] @ _dag(Um[xmm_pn]) @ _dag(Un[xmm]) @ Um[xmm]",
     "q = q + _dag(Um[xmm]) @ Un[xmm] @ Um[xmm_pn] @ _dag(Un[x])", pins.abelian_flux_error, 1e-10),
    ("dirac", "T -= kappa * csw", "T += kappa * csw", pins.abelian_flux_error, 1e-10),
    ("dirac", '"st,nab->nsatb"', '"st,nab->nastb"', pins.abelian_flux_error, 1e-10),
    ("gamma", "np.block([[Z2, -1j * PAULI[k]], [1j * PAULI[k], Z2]])",
     "np.block([[Z2, 1j * PAULI[k]], [-1j * PAULI[k], Z2]])", pins.free_field_error, 1e-10),
    ("evenodd", "return x_e - self.D_pp_inv(0, self.D_hop(0, t))", "return x_e - self.D_pp(0, self.D_hop(0, t))",
     pins.schur_dense_error, 1e-10),
    ("evenodd", "b_e - self.D_hop(0, self.D_pp_inv(1, b_o))", "b_e + self.D_hop(0, self.D_pp_inv(1, b_o))",
     lambda: pins.lu_vs_bicgstab_error(evenodd_solve=True, maxiter=400), 1e-10),
    ("evenodd", "x[lat.odd] = self.D_pp_inv(1, b[lat.odd] - self.D_hop(1, x_e))",
     "x[lat.odd] = self.D_pp_inv(1, b[lat.odd] + self.D_hop(1, x_e))",
     lambda: pins.lu_vs_bicgstab_error(evenodd_solve=True, maxiter=400), 1e-10),
    ("solvers", "x = x + alpha * p + omega * s", "x = x + alpha * p", lambda: pins.lu_vs_bicgstab_error(maxiter=400), 1e-10),
    ("solvers", "r = s - omega * t", "r = s + omega * t", lambda: pins.lu_vs_bicgstab_error(maxiter=400), 1e-10),
    ("solvers", "np.kron(_g.I4 + g, U[mu][y].conj().T)", "np.kron(_g.I4 + g, U[mu][y].conj())", pins.dense_vs_stencil_error, 1e-10),
    # Moebius domain wall
    ("domainwall", "out[s][:, LOWER] = up[:, LOWER]\n            out[s][:, UPPER] = dn[:, UPPER]",
     "out[s][:, UPPER] = up[:, UPPER]\n            out[s][:, LOWER] = dn[:, LOWER]", pins.mobius_overlap_error, 1e-10),
    ("domainwall", "up = psi[s + 1] if s + 1 < Ls else -mf * psi[0]", "up = psi[s + 1] if s + 1 < Ls else mf * psi[0]",
     pins.mobius_overlap_error, 1e-10),
    ("domainwall", "+ self.c * self.W(Ppsi[s], sites) - Ppsi[s][sites]", "- Ppsi[s][sites]",
     pins.mobius_overlap_error, 1e-10),
    ("domainwall", "return (4.0 - self.M5) * psi4[sites]", "return (4.0 + self.M5) * psi4[sites]",
     pins.mobius_free_field_error, 1e-10),
    ("domainwall", "- 0.5 * dirac.hop(self.U, psi4, lat, self.bc, sites)", "- dirac.hop(self.U, psi4, lat, self.bc, sites)",
     pins.mobius_free_field_error, 1e-10),
    ("domainwall", "Bv = _mix(self.B[0], self.B[1], v)", "Bv = v", pins.mobius_schur_dense_error, 1e-10),
    ("domainwall", "return x_e - self.D_pp_inv(self.D_hop(0, t))", "return x_e - self.D_pp(self.D_hop(0, t))",
     pins.mobius_schur_dense_error, 1e-10),
    ("domainwall", "S[s, Ls - 1] = -mf", "S[s, Ls - 1] = mf", pins.mobius_schur_dense_error, 1e-10),
    ("domainwall", "return _mix(self.Ainv[0].T, self.Ainv[1].T, v)", "return _mix(self.Ainv[0], self.Ainv[1], v)",
     pins.mobius_adjoint_error, 1e-10),
    ("domainwall", "return _mix(self.B[0].T, self.B[1].T, _g5(h))", "return _mix(self.B[0].T, self.B[1].T, h)",
     pins.mobius_adjoint_error, 1e-10),
    ("solvers", "p = r + (rr_new / rr) * p", "p = r", pins.cg_error, 1e-10),
    # two-level multigrid
    ("multigrid", "A[:, i] /= np.linalg.norm(A[:, i])", "A[:, i] /= 1.0", pins.mg_transfer_error, 1e-10),
    ("multigrid", "out[b, chi] = self.Q[b][chi].conj().T @", "out[b, chi] = self.Q[b][chi].T @", pins.mg_transfer_error, 1e-10),
    ("multigrid", "keep = (blocks.of_site[j] == blocks.of_site[x]) * np.where(wraps, bc[mu], 1.0)\n        chi = keep[:, None, None] * psi[j]\n        out -= kappa * np.einsum(\"st,ntc->nsc\", _g.I4 + g",
     "keep = (blocks.of_site[j] != blocks.of_site[x]) * np.where(wraps, bc[mu], 1.0)\n        chi = keep[:, None, None] * psi[j]\n        out -= kappa * np.einsum(\"st,ntc->nsc\", _g.I4 + g",
     pins.mg_block_operator_error, 1e-10),
    ("multigrid", "chi @ np.conj(U[mu][j])", "chi @ U[mu][j]", pins.mg_block_operator_error, 1e-10),
    ("multigrid", "alpha = np.vdot(q[s], rho[s]) / qq", "alpha = np.vdot(rho[s], q[s]) / qq", pins.mg_sap_error, 1e-10),
    ("multigrid", "for colour in (0, 1):\n                x = x + self.mr(b - self.D(x), colour, mr_steps)",
     "for colour in (1, 0):\n                x = x + self.mr(b - self.D(x), colour, mr_steps)", pins.mg_sap_error, 1e-10),
    ("multigrid", "x = x + self.mr(b - self.D(x), colour, mr_steps)", "x = x + self.mr(b, colour, mr_steps)",
     pins.mg_sap_error, 1e-10),
    ("multigrid", "return z + self.sap(r - self.D(z), cycles, mr_steps)", "return z + self.sap(r, cycles, mr_steps)",
     pins.mg_cycle_error, 1e-10),
    ("multigrid", "x = x + alpha * ph + omega * sh", "x = x + alpha * p + omega * s", pins.mg_solve_error, 1e-10),
    ("multigrid", "e[O] = np.linalg.solve(A_O, r[O] - H_OE @ e_E)", "e[O] = np.linalg.solve(A_O, r[O] + H_OE @ e_E)",
     pins.mg_coarse_evenodd_error, 1e-10),
    ("multigrid", "rhs = np.linalg.solve(A_E, r[E] - H_EO @ AOinv_rO)", "rhs = np.linalg.solve(A_E, r[E])",
     pins.mg_coarse_evenodd_error, 1e-10),
    # staggered
    ("staggered", "for nu in range(mu):", "for nu in range(mu + 1):", pins.staggered_free_field_error, 1e-10),
    ("staggered", "out -= 0.5 * e * np.einsum", "out += 0.5 * e * np.einsum", pins.staggered_free_field_error, 1e-10),
    ("staggered", "out += 0.5 * e * np.einsum(\"nab,nb->na\", U[mu][sites]", "out += e * np.einsum(\"nab,nb->na\", U[mu][sites]",
     pins.staggered_free_field_error, 1e-10),
    ("staggered", "_dag(U[mu][j]), ph * chi[j]", "U[mu][j], ph * chi[j]", pins.staggered_antihermitian_error, 1e-10),
    ("staggered", "np.einsum(\"nab,nb->na\", U[mu][sites], ph * chi[j])", "np.einsum(\"nba,nb->na\", U[mu][sites], ph * chi[j])",
     pins.staggered_covariance_error, 1e-10),
    ("staggered", "return self.m * b[lat.even] - self.D_hop(0, b[lat.odd])", "return self.m * b[lat.even] + self.D_hop(0, b[lat.odd])",
     pins.staggered_dense_error, 1e-10),
    ("staggered", "x[lat.odd] = (b[lat.odd] - self.D_hop(1, x_e)) / self.m", "x[lat.odd] = (b[lat.odd] - self.D_hop(1, x_e))",
     pins.staggered_dense_error, 1e-10),
    ("solvers", "alpha = rr / dot(p, Ap).real", "alpha = rr / dot(Ap, Ap).real", pins.cg_error, 1e-10),
]


def _load_mutant(modname, old, new):
    mod = importlib.import_module(f"oracle.{modname}")
    src = inspect.getsource(mod)
    assert src.count(old) >= 1, f"mutation anchor not found in oracle/{modname}.py: {old!r}"
    ns = {"__name__": f"oracle.{modname}_mutant", "__package__": "oracle"}
    exec(compile(src.replace(old, new, 1), f"oracle/{modname}.py(mutant)", "exec"), ns)
    return mod, ns


@pytest.mark.parametrize("case", range(len(MUTANTS)), ids=[f"{m[0]}:{m[2][:40]}" for m in MUTANTS])
def test_planted_mistake_is_caught(case, monkeypatch):
    modname, old, new, pin, threshold = MUTANTS[case]
    mod, ns = _load_mutant(modname, old, new)
    for name, obj in ns.items():
        if not name.startswith("__") and hasattr(mod, name) and (inspect.isfunction(obj) or inspect.isclass(obj) or name == "GAMMA"):
            monkeypatch.setattr(mod, name, obj)
    assert pin() > threshold


def test_unmutated_oracle_passes_every_pin_used_above():
    for _, _, _, pin, _ in MUTANTS:
        assert pin() < 1e-10
    assert oracle is not None
