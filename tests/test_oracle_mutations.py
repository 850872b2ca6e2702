"""The oracle's pins catch plausible mistakes planted in the oracle.

Each row below plants one mistake in a copy of `oracle/` (a dropped term, a
flipped sign, a wrong index, a wrong factor, a misread rule of the paper) and
names the pin that must then fail.  The copy lives in a temporary folder with
the tests beside it; the pin runs there in its own Python process, so the
repository's oracle is never touched.  A control run of every named pin on
the unchanged copy must pass first, so that a failure really comes from the
planted mistake.

Mistakes that change nothing the method computes are not listed: swapping
the order of the gradient components of the basis (K sums over them), a
floor on the trained diagonal of G that the training never reaches, or a
constant factor per parameter in the gradient that Adam receives (its step
divides the factor out).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

B = "tests/test_oracle_basis.py::"
S = "tests/test_oracle_sources.py::"
GEO = "tests/test_oracle_geometry.py::"
DI = "tests/test_oracle_discretize.py::"
I = "tests/test_oracle_integrators.py::"
P = "tests/test_oracle_pipeline.py::"
SC = "tests/test_oracle_schemes.py::"
A = "tests/test_oracle_adjoint.py::"
L = "tests/test_oracle_learned.py::"

# (oracle module, text as written, planted mistake, pin that must fail)
MISTAKES = [
    # GLL / Lagrange basis (Sec. Spatial discretization)
    ("basis.py", "w = 2.0 / (p * (p + 1) *", "w = 2.0 / (p * (p - 1) *", B + "test_gll_textbook_tables"),
    ("basis.py", "r = npleg.legroots(npleg.legder(cp))", "r = npleg.legroots(np.eye(p)[p - 1])",
     B + "test_gll_textbook_tables"),
    ("basis.py", "out[:, i] *= (xi - nodes[j]) / (nodes[i] - nodes[j])",
     "out[:, i] *= (xi - nodes[j]) / (nodes[j] - nodes[i])", B + "test_lagrange_properties"),
    ("basis.py", "term = np.full(len(xi), 1.0 / (nodes[i] - nodes[k]))",
     "term = np.full(len(xi), 1.0 / (nodes[k] - nodes[i]))", B + "test_lagrange_properties"),
    ("basis.py", "term *= (xi - nodes[j]) / (nodes[i] - nodes[j])", "term *= (xi - nodes[k]) / (nodes[i] - nodes[j])",
     B + "test_lagrange_properties"),
    # source terms (Eqs. ft, fx and the workloads' wavelets)
    ("sources.py", "    t0 = 1.0 / f0\n    a =", "    t0 = 1.5 / f0\n    a =", S + "test_ricker_closed_form"),
    ("sources.py", "(1.0 - 2.0 * a) * np.exp(-a)", "(1.0 - a) * np.exp(-a)", S + "test_ricker_closed_form"),
    ("sources.py", "return -(t - t0)", "return (t - t0)", S + "test_gaussian_derivative_eq_ft"),
    ("sources.py", "s = 1.0 / (2.0 * np.pi * fs)", "s = 1.0 / (np.pi * fs)", S + "test_gaussian_derivative_eq_ft"),
    ("sources.py", "np.where(t <= ncycles / fs, val, 0.0)", "np.where(t <= 1.0 / fs, val, 0.0)",
     S + "test_sine_burst"),
    ("sources.py", "np.sin(np.pi * fs * t / ncycles) ** 2", "np.sin(np.pi * fs * t / ncycles)", S + "test_sine_burst"),
    ("sources.py", "/ (2.0 * sigma * sigma))", "/ (sigma * sigma))", S + "test_bell_eq_fx"),
    # immersed geometry: point test and exact box classification
    ("geometry.py", "inside |= (((x - c) / a) ** 2).sum(axis=1) <= 1.0",
     "inside |= (np.abs((x - c) / a)).sum(axis=1) <= 1.0", GEO + "test_classify_matches_sampling"),
    ("geometry.py", "near = np.clip(0.0, slo, shi)", "near = slo", GEO + "test_classify_matches_sampling"),
    ("geometry.py", "far = np.maximum(np.abs(slo), np.abs(shi))", "far = np.abs(shi)",
     GEO + "test_classify_matches_sampling"),
    ("geometry.py", "if dmax2 <= 1.0:\n                return EMPTY", "if dmax2 <= 1.0:\n                cut = True",
     GEO + "test_classify_matches_sampling"),
    ("geometry.py", "if dmin2 < 1.0:\n                cut = True", "if dmin2 < 0.9:\n                cut = True",
     GEO + "test_classify_matches_sampling"),
    ("geometry.py", "return x[:, self.axis] < self.level", "return x[:, self.axis] > self.level",
     DI + "test_single_cell_quadtree_depth13"),
    # discretisation (Eqs. Mglobal, K, f; spacetree quadrature; partition)
    ("discretize.py", "    jac = np.prod(h / 2.0)\n    wq", "    jac = np.prod(h)\n    wq", DI + "test_assembly_invariants"),
    ("discretize.py", "basis.lagrange_deriv(nodes, xr[:, k]) * (2.0 / h[k])",
     "basis.lagrange_deriv(nodes, xr[:, k]) * (1.0 / h[k])", DI + "test_uncut_critical_time_step_table"),
    ("discretize.py", "(wq * rho * c * c)", "(wq * rho * c)", DI + "test_stiffness_scales_with_the_square_of_the_wave_speed"),
    ("discretize.py", "speed[uncut, None] ** 2 * Ke1", "speed[uncut, None] * Ke1",
     DI + "test_stiffness_scales_with_the_square_of_the_wave_speed"),
    ("discretize.py", "wts.append(np.prod([w1[i] for i in idx]))", "wts.append(np.sum([w1[i] for i in idx]))",
     DI + "test_single_cell_exact_split"),
    ("discretize.py", "out_w.append(ref_w * np.prod(half))", "out_w.append(ref_w)",
     DI + "test_physical_area_converges_to_analytic"),
    ("discretize.py", "out_x.append(rlo + (ref_pts + 1.0) * half)", "out_x.append(rlo + ref_pts * half)",
     DI + "test_single_cell_exact_split"),
    ("discretize.py", "if level < depth and geom", "if level <= depth and geom", DI + "test_single_cell_quadtree_depth13"),
    ("discretize.py", "aq = np.where(phys, 1.0, alpha)\n        fv", "aq = np.where(phys, alpha, 1.0)\n        fv",
     DI + "test_assembly_invariants"),
    ("discretize.py", "    xl, wl = basis.gll_points(p)\n    xr2", "    xl, wl = basis.gauss_points(p + 1)\n    xr2",
     DI + "test_uncut_critical_time_step_table"),
    ("discretize.py", "Me = (N * (wq * rho)[:, None]).T @ N", "Me = (N * (wr * rho)[:, None]).T @ N",
     DI + "test_assembly_invariants"),
    ("discretize.py", "if eta < EMPTY_FILL:", "if eta < 0.01:", DI + "test_empty_cell_threshold_is_fill_ratio_1e_10"),
    ("discretize.py", "fe = (fv * (wr * jac)[None, :]) @ Nq", "fe = (fv * wr[None, :]) @ Nq",
     DI + "test_load_vector_integrates_constant_and_linear_loads"),
    ("discretize.py", "fe = N.T @ (wq * fvals)", "fe = N.T @ (wr * fvals)",
     DI + "test_load_vector_integrates_constant_and_linear_loads"),
    ("discretize.py", "xq = lo[:, None, :] + (xr[None, :, :] + 1.0) / 2.0 * grid.h",
     "xq = lo[:, None, :] + (xr[None, :, :] + 1.0) * grid.h", DI + "test_load_vector_integrates_constant_and_linear_loads"),
    ("discretize.py", "fv = fx(lo + (xr + 1.0) / 2.0 * grid.h)", "fv = fx(lo + (xr + 1.0) * grid.h)",
     DI + "test_load_vector_integrates_constant_and_linear_loads"),
    ("discretize.py", "ids += (cells[:, k:k + 1] * grid.p + local[None, :, k]) * stride",
     "ids += (cells[:, k:k + 1] * grid.p + local[None, ::-1, k]) * stride",
     DI + "test_load_vector_integrates_constant_and_linear_loads"),
    ("discretize.py", "is_c[nodes[ctype == CUT].ravel()] = True", "is_c[nodes[ctype == CUT][:, :1].ravel()] = True",
     DI + "test_assembly_invariants"),
    ("discretize.py", "return 2.0 / np.sqrt(lam.max())", "return 1.0 / np.sqrt(lam.max())",
     DI + "test_uncut_critical_time_step_table"),
    # time integrators (Eqs. CDMstep, CDMacc, Newmark1, Newmark2; Fig. TrapCDMIMEX)
    ("integrators.py", "BETA = 0.25", "BETA = 0.5", I + "test_trapezoidal_single_mode_closed_form"),
    ("integrators.py", "GAMMA = 0.5", "GAMMA = 0.6", I + "test_trapezoidal_single_mode_closed_form"),
    ("integrators.py", "u_next = 2.0 * u - u_prev + dt * dt * a", "u_next = 2.0 * u - u_prev + 0.5 * dt * dt * a",
     I + "test_cdm_single_mode_closed_form"),
    ("integrators.py", "u_prev = u - dt * np.asarray(v0) + 0.5 * dt * dt * a0",
     "u_prev = u - dt * np.asarray(v0) - 0.5 * dt * dt * a0", I + "test_cdm_single_mode_closed_form"),
    ("integrators.py", "a0 = solve(ft(0.0) * fx - K @ u)", "a0 = solve(-(K @ u))",
     SC + "test_without_cut_cells_all_central_difference_forms_are_imex"),
    ("integrators.py", "        t = k * dt\n        a = solve", "        t = (k + 1) * dt\n        a = solve",
     SC + "test_without_cut_cells_all_central_difference_forms_are_imex"),
    ("integrators.py", "u_pred = u + dt * v + (0.5 - BETA) * dt * dt * a", "u_pred = u + dt * v + (0.5 + BETA) * dt * dt * a",
     I + "test_trapezoidal_single_mode_closed_form"),
    ("integrators.py", "        v = v_pred + GAMMA * dt * a", "        v = v_pred + BETA * dt * a",
     I + "test_trapezoidal_single_mode_closed_form"),
    ("integrators.py", "        t1 = (k + 1) * dt", "        t1 = k * dt", SC + "test_trapezoidal_is_imex_with_every_dof_implicit"),
    ("integrators.py", "a_c[self.Ic] = self.Mcc_lu.solve(self.ft(0.0) * self.fxc - self.Kc @ u)", "a_c[self.Ic] = 0.0",
     I + "test_imex_with_all_dofs_implicit_is_trapezoidal"),
    ("integrators.py", "v_c[self.Ic] = v[self.Ic]", "v_c[self.Ic] = 0.0", I + "test_spring_chain_imex_second_order"),
    ("integrators.py", "u_prev_d[self.Id] = u[self.Id] - dt * v[self.Id] + 0.5 * dt * dt * a0d",
     "u_prev_d[self.Id] = u[self.Id] - dt * v[self.Id]", I + "test_imex_with_no_implicit_dofs_is_cdm"),
    ("integrators.py", "a0d = (self.ft(0.0) * self.fxd - self.Kd @ u) / self.mdd",
     "a0d = (self.ft(0.0) * self.fxd - self.Kd @ u) / self.mdd.mean()", I + "test_imex_with_no_implicit_dofs_is_cdm"),
    ("integrators.py", "a_d = (self.ft(t_n) * self.fxd", "a_d = (self.ft(t_n1) * self.fxd",
     I + "test_spring_chain_imex_second_order"),
    ("integrators.py", "uc_pred = u[Ic] + dt * s.v_c[Ic] + (0.5 - BETA)", "uc_pred = u[Ic] + dt * s.v_c[Ic] + (1.0 - BETA)",
     I + "test_spring_chain_imex_second_order"),
    ("integrators.py", "vc_pred = s.v_c[Ic] + (1.0 - GAMMA) * dt * s.a_c[Ic]", "vc_pred = s.v_c[Ic]",
     I + "test_imex_with_all_dofs_implicit_is_trapezoidal"),
    ("integrators.py", "            u_pred = u_new.copy()", "            u_pred = u.copy()",
     I + "test_spring_chain_imex_second_order"),
    ("integrators.py", "        t_n1 = (s.n + 1) * dt", "        t_n1 = s.n * dt",
     SC + "test_trapezoidal_is_imex_with_every_dof_implicit"),
    ("integrators.py", "self.S_lu = spla.splu(_csc(Mcc + BETA * dt * dt * Kcc)", "self.S_lu = spla.splu(_csc(Mcc + GAMMA * dt * dt * Kcc)",
     I + "test_imex_with_all_dofs_implicit_is_trapezoidal"),
    ("integrators.py", "u_new[Ic] = uc_pred + BETA * dt * dt * ac", "u_new[Ic] = uc_pred + GAMMA * dt * dt * ac",
     I + "test_imex_with_all_dofs_implicit_is_trapezoidal"),
    ("integrators.py", "v_c[Ic] = vc_pred + GAMMA * dt * ac", "v_c[Ic] = vc_pred + BETA * dt * ac",
     I + "test_imex_with_all_dofs_implicit_is_trapezoidal"),
    # one workload end to end: time-step rule, independent columns
    ("pipeline.py", "dt = dt_factor * uncut_critical_dt(p, grid.h, rho, cmax)",
     "dt = dt_factor * uncut_critical_dt(p, grid.h, rho, c0)", P + "test_time_step_rule_takes_the_fastest_uncut_cell"),
    ("pipeline.py", "return [setup(src_pos=pos[k:k + 1], **kw) for k in range(len(pos))]",
     "return [setup(src_pos=pos[:1], **kw) for k in range(len(pos))]",
     P + "test_independent_columns_superpose_to_the_multi_source_run"),
    # comparison schemes (Eqs. HRZ; Table criticaltimestepsizes)
    ("schemes.py", "return np.diag(d * (Me.sum() / d.sum()))", "return np.diag(d)", SC + "test_hrz_textbook_bar_elements"),
    ("schemes.py", "return np.diag(d * (Me.sum() / d.sum()))", "return np.diag(Me.sum(axis=1))",
     SC + "test_hrz_keeps_the_diagonal_shape_unlike_row_sums"),
    ("schemes.py", "Mt = hrz_lump(Me) if d.cell_type[cid] == CUT else Me\n        np.add.at", "Mt = Me\n        np.add.at",
     SC + "test_assembled_hrz_mass"),
    ("schemes.py", "dt_u = 2.0 / np.sqrt(lam_u)", "dt_u = 1.0 / np.sqrt(lam_u)", SC + "test_element_eigenvalue_bound"),
    ("schemes.py", "lam = sla.eigh(Ke, Mt, eigvals_only=True)[-1]", "lam = sla.eigh(Ke, Mt, eigvals_only=True)[0]",
     SC + "test_element_eigenvalue_bound"),
    # discrete adjoint of the IMEX step
    ("adjoint.py", "dK = 2.0 * cell_c[cid] * Ke1", "dK = cell_c[cid] * Ke1", A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "abar_c = abar[Ic] + BETA * dt * dt * ubar[Ic] + GAMMA * dt * vbar[Ic]",
     "abar_c = abar[Ic] + BETA * dt * dt * ubar[Ic]", A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "ubar_n[Id] += 2.0 * ubar_d_next + ubar_prev_d[Id]", "ubar_n[Id] += 2.0 * ubar_d_next",
     A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "w2[Ic] += BETA * dt * dt * a1", "w2[Ic] += 0.0 * a1", A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "abar_n[Ic] = (0.5 - BETA) * dt * dt * ubar_cp + (1.0 - GAMMA) * dt * vbar_cp",
     "abar_n[Ic] = (0.5 - BETA) * dt * dt * ubar_cp", A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "us = [h[0] for h in hist[1:]] + [last]", "us = [h[0] for h in hist]",
     A + "test_adjoint_gradient_matches_central_differences"),
    ("adjoint.py", "J += 0.5 * float(e @ e)\n    cells", "J += float(e @ e)\n    cells",
     A + "test_adjoint_gradient_matches_central_differences"),
    # PCG, FSAI, Kaporin, Adam and the learned start
    ("learned.py", "p = z + (rz_new / rz) * p", "p = z + (rz / rz_new) * p", L + "test_pcg_matches_direct_solve"),
    ("learned.py", "alpha = rz / (p @ q)", "alpha = rz / (p @ p)", L + "test_pcg_matches_direct_solve"),
    ("learned.py", "        res = np.linalg.norm(r) / nb\n        if res <= tol:", "        res = np.linalg.norm(r)\n        if res <= tol:",
     L + "test_learned_preconditioner_shortens_cg_on_the_methods_systems"),
    ("learned.py", "return G @ (G.T @ r)", "return G.T @ (G @ r)", L + "test_exact_inverse_factor_has_zero_loss_and_one_pcg_step"),
    ("learned.py", "grad = np.sum(D[rows] * Z[indices] + R[rows] * Q[indices], axis=1)",
     "grad = np.sum(D[rows] * Z[indices] + R[indices] * Q[rows], axis=1)", L + "test_fsai_gradient_matches_central_differences"),
    ("learned.py", "grad[diag] -= 2.0 / vals[diag]", "grad[diag] -= 1.0 / vals[diag]",
     L + "test_kaporin_gradient_matches_central_differences"),
    ("learned.py", "loss = float(np.dot(vals, sg) - 2.0 * np.sum(np.log(vals[diag])))",
     "loss = float(np.dot(vals, sg) - np.sum(np.log(vals[diag])))", L + "test_kaporin_gradient_matches_central_differences"),
    ("learned.py", "vals[ks] = y / np.sqrt(y[Q == j][0])", "vals[ks] = y / y[Q == j][0]",
     L + "test_kaporin_minimiser_is_the_closed_form_fsai"),
    ("learned.py", "mhat = m / (1.0 - beta1 ** t)", "mhat = m", L + "test_adam_first_step_closed_form"),
    ("learned.py", "vhat = v / (1.0 - beta2 ** t)", "vhat = v", L + "test_adam_first_step_closed_form"),
    ("learned.py", "vals[k] = 1.0 / np.sqrt(d[i])", "vals[k] = 1.0 / d[i]",
     L + "test_learned_preconditioner_shortens_cg_on_the_methods_systems"),
    ("learned.py", "grad = np.array([float(np.sum(2.0 * wt *", "grad = np.array([float(np.sum(1.0 * wt *",
     L + "test_extrapolation_gradient_matches_central_differences"),
    ("learned.py", "H = np.stack([A[:, s - k] for k in range(K)])", "H = np.stack([A[:, s - k - 1] for k in range(K)])",
     L + "test_extrapolation_exact_on_quadratic_sequences"),
]


def _copy_tree(base):
    ignore = shutil.ignore_patterns("__pycache__", "*.pyc")
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(base, "oracle"), ignore=ignore)
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(base, "tests"), ignore=ignore)
    pkg = os.path.join(base, "paper_2310_14712_gb300")
    os.makedirs(pkg)
    for name in ("__init__.py", "workloads.py"):        # the seeded inputs only
        shutil.copy(os.path.join(ROOT, "paper_2310_14712_gb300", name), pkg)


def _run_pins(base, pins):
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    env["PYTHONDONTWRITEBYTECODE"] = "1"
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *pins],
                       cwd=base, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout + r.stderr


def _planted(k):
    module, before, after, pin = MISTAKES[k]
    base = tempfile.mkdtemp(prefix="oracle_mistake_")
    try:
        _copy_tree(base)
        path = os.path.join(base, "oracle", module)
        with open(path) as f:
            src = f.read()
        if src.count(before) != 1:
            return k, None, f"{module}: the text to change occurs {src.count(before)} times"
        with open(path, "w") as f:
            f.write(src.replace(before, after))
        rc, out = _run_pins(base, [pin])
        return k, rc, out
    finally:
        shutil.rmtree(base, ignore_errors=True)


def test_every_planted_mistake_fails_its_pin():
    pins = sorted({m[3] for m in MISTAKES})
    base = tempfile.mkdtemp(prefix="oracle_control_")
    try:
        _copy_tree(base)
        rc, out = _run_pins(base, pins)
    finally:
        shutil.rmtree(base, ignore_errors=True)
    assert rc == 0, "the pins fail on the unchanged oracle:\n" + out[-2000:]

    workers = max(1, min(8, os.cpu_count() or 1))
    missed = []
    with cf.ThreadPoolExecutor(workers) as ex:
        for k, rc, out in ex.map(_planted, range(len(MISTAKES))):
            module, _, after, pin = MISTAKES[k]
            # exit code 1: the pin ran and failed (not a collection or usage error)
            if rc != 1 or "failed" not in out.splitlines()[-1]:
                missed.append(f"{module}: {after!r} -> {pin} (exit {rc})\n{out[-600:]}")
    assert not missed, "planted mistakes that no pin caught:\n" + "\n".join(missed)


def test_mistake_table_names_existing_pins():
    for module, before, after, pin in MISTAKES:
        path, name = pin.split("::")
        with open(os.path.join(ROOT, path)) as f:
            assert f"def {name}(" in f.read(), pin
        with open(os.path.join(ROOT, "oracle", module)) as f:
            assert f.read().count(before) == 1, (module, before)
        assert before != after
