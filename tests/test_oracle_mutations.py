"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in
the oracle's own source on the CPU (a changed constant, a flipped sign, a
dropped factor, an index or operand swapped, the wrong branch of a formula),
rebuilds the patched function from that source, and runs one pin from the
`test_oracle_*` modules against it: the pin must fail.  The unpatched oracle
passes every one of these pins in its own module."""
import importlib
import inspect
import sys
import textwrap

import pytest

from oracle import adjoint, delta, fsi, helmholtz, mac, schur, step

# (case, owner of the function, function, text in its source, planted text,
#  pin module, pin function, pin arguments)
MUTATIONS = [
    ("phi inner branch constant", delta, "phi", "1.0 - 3.0 * ri * ri", "1.0 - 2.0 * ri * ri",
     "test_oracle_delta", "test_phi_closed_form_values", ()),
    ("phi outer branch slope", delta, "phi", "(5.0 - 3.0 * ro", "(5.0 - 2.5 * ro",
     "test_oracle_delta", "test_phi_moments", (0.13,)),
    ("R: face and centre offsets swapped", delta, "_regularization",
     "offset = 0.0 if e == d else 0.5", "offset = 0.5 if e == d else 0.0",
     "test_oracle_delta", "test_linear_field_interpolated_exactly", ()),
    ("R: y weights taken from the z axis", delta, "_regularization",
     "w[2][:, :, None, None] * w[1][:, None, :, None]",
     "w[2][:, :, None, None] * w[2][:, None, :, None]",
     "test_oracle_delta", "test_interp_matches_bruteforce_and_adjoint", ()),
    ("dR/dX: sign of phi'", delta, "_regularization",
     "w.append(-phi_prime(dist) / h)", "w.append(phi_prime(dist) / h)",
     "test_oracle_adjoint", "test_regularization_derivative_central_difference", (0,)),
    ("phi': inner branch sign", delta, "phi_prime", "out[inner] = -ri /", "out[inner] = ri /",
     "test_oracle_adjoint", "test_phi_prime_central_difference", ()),
    ("G: minus-side coefficient", mac, "gradient_matrix",
     "np.full(f.size, -1.0 / g.h)", "np.full(f.size, -0.5 / g.h)",
     "test_oracle_mac", "test_gradient_kills_constants", ()),
    ("G^T: minus-side sign", mac, "apply_GT", "out[tuple(minus)] -= fi",
     "out[tuple(minus)] += fi",
     "test_oracle_mac", "test_matrix_free_operators_match_matrices", ()),
    ("G: cells on the wrong side", mac, "apply_G", "np.diff(p3, axis=axis) / g.h",
     "-np.diff(p3, axis=axis) / g.h",
     "test_oracle_mac", "test_matrix_free_operators_match_matrices", ()),
    ("L eigenvalues: wrong wavenumbers", mac, "neumann_eigenvalues", "np.pi * k / n",
     "np.pi * k / (n + 1)", "test_oracle_mac", "test_neumann_eigenvalues", ()),
    ("L^+: constant mode kept", mac, "laplacian_pinv", "rh[0, 0, 0] = 0.0",
     "rh[0, 0, 0] = rh[0, 0, 0]",
     "test_oracle_mac", "test_pinv_matches_dense_pseudoinverse", ()),
    ("S~ apply: factor 2 dropped", schur.SchurSystem, "apply_S_tilde",
     "+ 2.0 * self.apply_BT", "+ 1.0 * self.apply_BT",
     "test_oracle_schur", "test_fgmres_matches_dense_bruteforce", ()),
    ("S~ dense: factor 2 dropped", schur.SchurSystem, "dense_S_tilde", "2.0 * (B.T @ B)",
     "1.0 * (B.T @ B)", "test_oracle_schur", "test_scalar_approximation_spectrum_like_table2",
     ()),
    ("S exact: C^-1 replaced by C", schur.SchurSystem, "dense_S_exact",
     "np.linalg.solve(Cd, Bd)", "(Cd @ Bd)",
     "test_oracle_schur", "test_schur_elimination_matches_block_saddle_solve", ()),
    ("saddle: sign of the (2,2) block", schur.SchurSystem, "saddle_matrix",
     "-self.C.toarray()", "self.C.toarray()",
     "test_oracle_schur", "test_schur_elimination_matches_block_saddle_solve", ()),
    ("b: factor 2 of B^T RHS_F dropped", schur.SchurSystem, "rhs_scalar",
     "+ 2.0 * self.apply_BT(rhs_F)", "+ self.apply_BT(rhs_F)",
     "test_oracle_step", "test_post_update_identities", ("scalar",)),
    ("F': factor 2 dropped", schur.SchurSystem, "force_scalar", "2.0 * (self.apply_B(p)",
     "(self.apply_B(p)", "test_oracle_step", "test_post_update_identities", ("scalar",)),
    ("update: dt/3 in place of 2dt/3", step, "step", "(2.0 * dt / 3.0) * (-mac.apply_G",
     "(dt / 3.0) * (-mac.apply_G", "test_oracle_step", "test_post_update_identities",
     ("exact",)),
    ("RHS_F: U^Gamma added", step, "step", "sys.R.T @ u_star - U_gamma",
     "sys.R.T @ u_star + U_gamma", "test_oracle_step", "test_post_update_identities",
     ("exact",)),
    ("predictor: BDF2 weight of u^n", step, "predictor_rhs", "(4.0 * u_n - u_nm1)",
     "(3.0 * u_n - u_nm1)", "test_oracle_step", "test_linear_in_time_solution_is_reproduced",
     (False,)),
    ("predictor: BDF2 weight of u^{n-1} dropped", step, "predictor_rhs",
     "(4.0 * u_n - u_nm1)", "(4.0 * u_n - 0.0 * u_nm1)",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (False,)),
    ("predictor: history levels swapped", step, "predictor_rhs", "(4.0 * u_n - u_nm1)",
     "(4.0 * u_nm1 - u_n)", "test_oracle_step", "test_linear_in_time_solution_is_reproduced",
     (False,)),
    ("predictor: dt in place of 2 dt", step, "predictor_rhs", "/ (2.0 * dt)", "/ dt",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (False,)),
    ("predictor: sign of G p^n", step, "predictor_rhs", "- mac.apply_G(g, p_n)",
     "+ mac.apply_G(g, p_n)", "test_oracle_step", "test_linear_in_time_solution_is_reproduced",
     (False,)),
    ("predictor: sign of R F^n", step, "predictor_rhs", "+ RF_n +", "- RF_n +",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (False,)),
    ("predictor: body force dropped", step, "predictor_rhs", "+ f_body", "+ 0.0 * f_body",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (False,)),
    ("predictor: sign of the convective term", step, "predictor_rhs",
     "rhs = rhs - advection(g, u_n)", "rhs = rhs + advection(g, u_n)",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (True,)),
    ("predictor: sign of the convective term (analytic pin)", step, "predictor_rhs",
     "rhs = rhs - advection(g, u_n)", "rhs = rhs + advection(g, u_n)",
     "test_oracle_step", "test_convective_term_drives_the_step_with_minus_sign", ()),
    ("predictor: convective term at u^{n-1}", step, "predictor_rhs",
     "rhs = rhs - advection(g, u_n)", "rhs = rhs - advection(g, u_nm1)",
     "test_oracle_step", "test_linear_in_time_solution_is_reproduced", (True,)),
    ("advection: one-sided centre value", step, "advection",
     "cc = 0.5 * (ud[tuple(lo)] + ud[tuple(hi)])", "cc = ud[tuple(hi)]",
     "test_oracle_step", "test_advection_conserves_energy_for_divergence_free_fields", ()),
    ("Helmholtz: wall ghost sign", helmholtz, "apply", "vm[tuple(sl)] = -v[tuple(sl)]",
     "vm[tuple(sl)] = v[tuple(sl)]",
     "test_oracle_helmholtz", "test_apply_matches_assembled_matrix", ()),
    ("Helmholtz solve: Neumann wavenumbers", helmholtz, "_eig_1d",
     "k = np.arange(1, n + 1)", "k = np.arange(0, n)",
     "test_oracle_helmholtz", "test_solve_matches_sparse_direct", ()),
    ("Rodrigues: Euler angle in place of AB2", fsi, "rodrigues_increment",
     "1.5 * nrm - 0.5 *", "1.0 * nrm - 0.0 *",
     "test_oracle_fsi", "test_rodrigues_increment_rotates_by_the_ab2_angle", ()),
    ("rigid update: buoyancy factor dropped", fsi, "rigid_velocities",
     "(th - 1.0) / th * g", "g", "test_oracle_fsi", "test_rigid_update_free_fall_is_exact",
     ()),
    ("volume fraction: outside counted", fsi, "volume_fraction",
     "num += np.maximum(-phi, 0.0)", "num += np.maximum(phi, 0.0)",
     "test_oracle_fsi", "test_volume_fraction_second_order", ()),
    ("enclosed angular momentum: z sign", fsi, "fluid_momentum",
     "ang[2] += np.sum(r[0] * w * e[1] - r[1] * w * e[0])",
     "ang[2] += np.sum(r[1] * w * e[0] - r[0] * w * e[1])",
     "test_oracle_fsi", "test_fluid_momentum_uniform_and_rotating_fields", ()),
    ("skew matrix: one sign", fsi, "skew", "[v[2], 0.0, -v[0]]", "[-v[2], 0.0, -v[0]]",
     "test_oracle_fsi", "test_rodrigues_increment_rotates_by_the_ab2_angle", ()),
    ("spread criterion: norm of F in place of F'", fsi, "fsi_step",
     "ratio = np.abs(sys.R @ Fc).sum() / nF", "ratio = np.abs(sys.R @ F).sum() / nF",
     "test_oracle_fsi", "test_spread_criterion_stops_early_with_the_same_body_motion", ()),
    ("two-way correction: half the update", fsi, "fsi_step",
     "u = u + xi * (1.0 / a) *", "u = u + xi * (0.5 / a) *",
     "test_oracle_fsi", "test_fixed_body_one_correction_equals_one_way_step", ()),
    ("body position: Euler step in place of BDF2", fsi, "fsi_step",
     "(2.0 / 3.0) * dt * b.us", "dt * b.us",
     "test_oracle_fsi", "test_corrections_approach_the_constrained_fixed_point", ()),
    ("FGMRES: update from V in place of Z", schur, "fgmres", "x = x + Z[:j_used].T @ y",
     "x = x + V[:j_used].T @ y",
     "test_oracle_schur", "test_fgmres_matches_dense_bruteforce", ()),
    ("FGMRES: projection on V_0 only", schur, "fgmres", "H[i, j] = np.dot(w, V[i])",
     "H[i, j] = np.dot(w, V[0])",
     "test_oracle_schur", "test_fgmres_matches_dense_bruteforce", ()),
    ("Helmholtz solve: sign of the viscous term", helmholtz, "solve",
     "r = r / (a + nu * lam)", "r = r / (a - nu * lam)",
     "test_oracle_helmholtz", "test_solve_matches_sparse_direct", ()),
    ("torque: lever and force swapped", step, "body_force_torque", "np.cross(r.T, f.T)",
     "np.cross(f.T, r.T)", "test_oracle_step", "test_body_force_torque_closed_form", ()),
    ("adjoint: a term of the chain dropped", adjoint, "step_vjp",
     "pairs.append((Gp, -2.0 * sys.apply_B(lam)))",
     "pairs.append((Gp, 0.0 * sys.apply_B(lam)))",
     "test_oracle_adjoint", "test_center_gradient_central_difference", (False,)),
    ("adjoint: sign of dJ/dU", adjoint, "step_vjp", "U_bar = -a * rhsF_bar",
     "U_bar = a * rhsF_bar", "test_oracle_adjoint", "test_U_gradient_exact_by_linearity",
     (False,)),
    ("adjoint: factor 2 of B lambda dropped", adjoint, "step_vjp",
     "rhsF_bar = rhsF_bar + 2.0 * sys.apply_B(lam)", "rhsF_bar = rhsF_bar + sys.apply_B(lam)",
     "test_oracle_adjoint", "test_U_gradient_exact_by_linearity", (False,)),
    ("force/torque VJP: cross product order", adjoint, "body_force_torque_vjp",
     "np.cross(wT, r.T).T", "np.cross(r.T, wT).T",
     "test_oracle_adjoint", "test_body_force_torque_vjp_central_difference", ()),
]


def _plant(monkeypatch, owner, name, old, new):
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (name, old)
    ns = dict(vars(sys.modules[fn.__module__]))
    exec(compile(src.replace(old, new), f"<planted {fn.__module__}.{name}>", "exec"), ns)
    monkeypatch.setattr(owner, name, ns[name])


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(monkeypatch, case):
    _, owner, name, old, new, pin_mod, pin_name, args = case
    pin = getattr(importlib.import_module(pin_mod), pin_name)
    _plant(monkeypatch, owner, name, old, new)
    with pytest.raises((AssertionError, ValueError)):
        pin(*args)


@pytest.mark.parametrize("case", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_rebuilt_unchanged_source_passes_the_pin(monkeypatch, case):
    # control: the same rebuild with nothing planted leaves the pin green, so
    # a failure above comes from the planted mistake, not from the rebuild
    _, owner, name, old, _, pin_mod, pin_name, args = case
    pin = getattr(importlib.import_module(pin_mod), pin_name)
    _plant(monkeypatch, owner, name, old, old)
    pin(*args)
