"""Mutation check of the oracle's pins (no GPU).

Each case plants one plausible mistake in a copy of oracle/soc.py: a wrong sign, a dropped
term, a shifted index, a swapped operand or axis, or a misread definition. The copy loads
as a separate module, and the pin named beside the mistake (a test of
tests/test_oracle_pins.py, run against the copy) must fail on it. The unmodified copy
passes every named pin. So each of these mistakes would be visible in the oracle, which
is fixed by the paper's numbers, closed forms, identities, symmetries and brute force
rather than by itself.

A pin fails by an assertion, by the oracle's own non-convergence error, or, for a mistake
that makes an iteration diverge, by no longer finishing within a limit far above its
normal run time. Any other exception means the planted edit itself is broken, and the
case fails.
"""
import os
import signal
import sys
import types

import pytest

import tests.test_oracle_pins as pins

SOURCE_PATH = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "oracle", "soc.py")


class PinTimeout(Exception):
    pass


# (name, [(text in oracle/soc.py, replacement)], pin, pin arguments, time limit in s or None)
CHANNEL = dict(D=4e-10, inlet_bc="face", k0=1e-6, m=0.7, h=1.25e-6)
CHANNEL_COARSE = dict(CHANNEL, h=5e-6)
ADJ = dict(objective="I_tot", kmode=0)
MUTATIONS = [
    # transport operator (Eq. nernst-planck-soc, face by face)
    ("advection_downwind",
     [("add(a, a, -pos); add(c, a, pos)", "add(a, c, -pos); add(c, c, pos)")],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL, None),
    ("x_diffusion_dropped",
     [("interior_faces(idx[:, :, :-1], idx[:, :, 1:], p.U[:, :, 1:-1],\n"
       "                   fluid[:, :, :-1] & fluid[:, :, 1:])",
       "interior_faces(idx[:, :, :-1], idx[:, :, 1:], p.U[:, :, 1:-1],\n"
       "                   np.zeros_like(fluid[:, :, 1:]))")],
     "test_xy_transposition_symmetry", {}, None),
    ("diffusion_coupling_sign",
     [("add(a, a, -dd); add(a, c, dd)", "add(a, a, -dd); add(a, c, -dd)")],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL, None),
    ("diffusion_scaled_by_h_not_h2",
     [("dd = np.where(both, D / (h * h), 0.0)", "dd = np.where(both, D / h * 8e5, 0.0)")],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL_COARSE, None),
    ("z_faces_shifted_by_one",
     [("interior_faces(idx[:-1], idx[1:], p.W[1:-1], fluid[:-1] & fluid[1:])",
       "interior_faces(idx[:-1], idx[1:], p.W[:-2], fluid[:-1] & fluid[1:])")],
     "test_uniform_state_is_steady_without_reaction", {}, None),
    ("velocity_scale_not_on_interior_faces",
     [("a, c, u, both = a.ravel(), c.ravel(), u.ravel() * beta, both.ravel()",
       "a, c, u, both = a.ravel(), c.ravel(), u.ravel(), both.ravel()")],
     "test_oracle_adjoint_matches_central_differences", ADJ, None),
    ("inlet_face_taken_as_ghost_cell",
     [('g = 2.0 if p.inlet_bc == "face" else 1.0\n    gd',
       'g = 1.0 if p.inlet_bc == "face" else 1.0\n    gd')],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL, None),
    ("inlet_value_not_s_in",
     [("np.add.at(b, cin, np.maximum(w, 0.0) / h * s_in)",
       "np.add.at(b, cin, np.maximum(w, 0.0) / h * 0.5)")],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL, None),
    ("outlet_outflow_dropped",
     [("add(cout, cout, -w / h)", "add(cout, cout, 0.0 * w / h)")],
     "test_uniform_state_is_steady_without_reaction", {}, None),
    ("outlet_outflow_sign",
     [("add(cout, cout, -w / h)", "add(cout, cout, w / h)")],
     "test_1d_channel_exact_discrete_closed_form", CHANNEL, None),
    # kinetics (Sec. II.B-II.D)
    ("thermal_voltage_at_273K",
     [("V_T = R_GAS * T / FARADAY", "V_T = R_GAS * 273.15 / FARADAY")],
     "test_kinetics_values_printed_in_paper", {}, None),
    ("reducing_voltage_sign",
     [("    V_ar = -eta\n", "    V_ar = eta\n")],
     "test_kinetics_values_printed_in_paper", {}, None),
    ("electron_count_dropped",
     [("Vt = n_e * V_ar / V_T", "Vt = V_ar / V_T")],
     "test_kinetics_values_printed_in_paper", {}, None),
    ("equilibrium_sigmoid_sign",
     [("s_eq = 1.0 / (1.0 + math.exp(-Vt))", "s_eq = 1.0 / (1.0 + math.exp(Vt))")],
     "test_affine_rate_law_matches_butler_volmer_form", dict(eta=-0.1, alpha=0.5), None),
    ("transfer_coefficient_swapped",
     [("A = math.exp(alpha * Vt)", "A = math.exp((1.0 - alpha) * Vt)")],
     "test_affine_rate_law_matches_butler_volmer_form", dict(eta=-0.1, alpha=0.3), None),
    ("rate_slope_exponent_sign",
     [("B = A * (1.0 + math.exp(-Vt))", "B = A * (1.0 + math.exp(Vt))")],
     "test_conservation_identity_any_state", {}, None),
    ("uniform_eta_backward_exponent",
     [("    return s ** alpha * (1.0 - s) ** (1.0 - alpha) * (math.exp(alpha * etat) -\n"
       "                                                     math.exp((alpha - 1.0) * etat))",
       "    return s ** alpha * (1.0 - s) ** (1.0 - alpha) * (math.exp(alpha * etat) -\n"
       "                                                     math.exp((1.0 - alpha) * etat))")],
     "test_uniform_eta_rate_is_the_butler_volmer_source", {}, None),
    ("uniform_eta_powers_swapped",
     [("    return s ** alpha * (1.0 - s) ** (1.0 - alpha) * (math.exp(alpha * etat) -\n"
       "                                                     math.exp((alpha - 1.0) * etat))",
       "    return s ** (1.0 - alpha) * (1.0 - s) ** alpha * (math.exp(alpha * etat) -\n"
       "                                                     math.exp((alpha - 1.0) * etat))")],
     "test_uniform_eta_rate_is_the_butler_volmer_source", {}, None),
    ("uniform_eta_slope_sign",
     [("s ** (alpha - 1.0) * (1.0 - s) ** (-alpha) * (alpha - s)",
       "s ** (alpha - 1.0) * (1.0 - s) ** (-alpha) * (s - alpha)")],
     "test_uniform_eta_slope_matches_central_differences", {}, None),
    # reactive area a_c = m_c n_wall / h
    ("side_walls_counted_as_fiber",
     [("    n[:-1] += s[1:]\n    return n",
       "    n[:-1] += s[1:]\n    n[:, :, 0] += 1\n    n[:, :, -1] += 1\n    return n")],
     "test_n_wall_brute_force", {}, None),
    ("z_neighbours_not_counted",
     [("    n[1:] += s[:-1]\n    n[:-1] += s[1:]\n", "\n")],
     "test_n_wall_brute_force", {}, None),
    ("area_per_volume_over_h2",
     [("kappa = np.where(fluid.ravel(), p.k0 * m * nw.ravel() / h, 0.0)",
       "kappa = np.where(fluid.ravel(), p.k0 * m * nw.ravel() / (h * h) * 1.25e-6, 0.0)")],
     "test_plug_flow_continuum_limit_first_order", {}, None),
    # residual and outputs (Sec. II.C)
    ("tau_inverted",
     [("tau = Vf / Q if Q > 0", "tau = Q / Vf * 1e-6 if Q > 0")],
     "test_residual_is_tau_times_rms_with_tau_the_residence_time", {}, None),
    ("residual_norm_not_rms",
     [("return op.tau * math.sqrt(float(np.mean(r * r))) if r.size else 0.0",
       "return op.tau * math.sqrt(float(np.sum(r * r))) if r.size else 0.0")],
     "test_residual_is_tau_times_rms_with_tau_the_residence_time", {}, None),
    ("current_sign",
     [("I_tot = scale * h ** 3 * float(np.sum(source(op, s)))",
       "I_tot = -scale * h ** 3 * float(np.sum(source(op, s)))")],
     "test_conservation_identity_any_state", {}, None),
    ("inlet_flux_without_diffusion",
     [("F_in = scale * h * h * (adv_in + dif_in)", "F_in = scale * h * h * adv_in")],
     "test_conservation_identity_any_state", {}, None),
    ("outlet_flux_on_inlet_plane",
     [("F_out = scale * h * h * float(np.sum(np.where(fout, w_out * s3[-1], 0.0)))",
       "F_out = scale * h * h * float(np.sum(np.where(fout, w_out * s3[0], 0.0)))")],
     "test_conservation_identity_any_state", {}, None),
    ("utilisation_without_inlet_state",
     [("denom = scale * op.Q * (1.0 - p.s_in)\n    U =", "denom = scale * op.Q\n    U =")],
     "test_steady_state_mass_balance_and_bounds", {}, None),
    # U_mt (Eq. umt-def)
    ("umt_electrode_cells_at_zero",
     [("fixed[elec] = 1.0", "fixed[elec] = 0.0")],
     "test_umt_closed_form_of_a_channel_inside_electrode_cells", dict(inlet_bc="face"), None),
    ("umt_keeps_the_inlet_value",
     [('s_in = 0.0 if mode == "umt" else p.s_in', "s_in = p.s_in")],
     "test_umt_closed_form_of_a_channel_inside_electrode_cells", dict(inlet_bc="face"), None),
    ("umt_unweighted_outlet_mean",
     [("return float(np.sum(np.where(fout, w * s3[-1], 0.0))) / "
       "float(np.sum(np.where(fout, w, 0.0)))",
       "return float(np.mean(s3[-1][fout]))")],
     "test_umt_closed_form_of_a_channel_inside_electrode_cells", dict(inlet_bc="ghost"), None),
    # kinetics mode 1: Newton's method with pseudo-transient continuation
    ("jacobian_without_reaction_slope",
     [("    d[k] = op.kappa[k] * rate_uniform_slope(s[k], op.kin.Vt, op.kin.alpha)\n"
       "    return (op.L + sp.diags(d)).tocsr()",
       "    d[k] = 0.0 * op.kappa[k] * rate_uniform_slope(s[k], op.kin.Vt, op.kin.alpha)\n"
       "    return (op.L + sp.diags(d)).tocsr()")],
     "test_oracle_adjoint_matches_central_differences", dict(objective="I_tot", kmode=1), None),
    ("pseudo_time_term_sign",
     [("A = (sp.diags(d / delta) - J).tocsr() if delta < 1e15 else -J",
       "A = (sp.diags(-d / delta) - J).tocsr() if delta < 1e15 else -J")],
     "test_uniform_eta_channel_without_diffusion_is_solved_cell_by_cell", dict(alpha=0.5), None),
    # steady state and the explicit loop (Algorithm 7)
    ("steady_state_source_sign",
     [("rhs_u = -(op.b[u] + op.L[u] @ op.fixed)", "rhs_u = (op.b[u] + op.L[u] @ op.fixed)")],
     "test_dense_lu_brute_force_small_lattice", {}, None),
    ("explicit_step_sign",
     [("            s[j] = s[i] + dt * rhs(op, s[i])", "            s[j] = s[i] - dt * rhs(op, s[i])")],
     "test_explicit_iteration_reaches_the_steady_state", dict(local_dt=True), 5.0),
    ("local_step_times_diagonal",
     [("        dt = np.where(u, cfl / np.where(d > 0, d, 1.0), 0.0)\n    else:\n"
       "        dt = np.where(u, dt_global(op, cfl), 0.0)\n    s = [",
       "        dt = np.where(u, cfl * np.where(d > 0, d, 1.0), 0.0)\n    else:\n"
       "        dt = np.where(u, dt_global(op, cfl), 0.0)\n    s = [")],
     "test_explicit_iteration_reaches_the_steady_state", dict(local_dt=True), 5.0),
    # discrete adjoint
    ("adjoint_operator_not_transposed",
     [("lam[u] = spla.spsolve(Luu.T.tocsc(), -g[u])", "lam[u] = spla.spsolve(Luu.tocsc(), -g[u])")],
     "test_oracle_adjoint_matches_central_differences", ADJ, None),
    ("adjoint_direct_term_dropped",
     [("        dm = (scale + lam) * kap0 * R\n", "        dm = lam * kap0 * R\n")],
     "test_oracle_adjoint_matches_central_differences", ADJ, None),
    ("adjoint_velocity_scale_sign",
     [("dbeta = float(np.dot(lam[u], adv_rhs[u])) / p.beta",
       "dbeta = -float(np.dot(lam[u], adv_rhs[u])) / p.beta")],
     "test_oracle_adjoint_matches_central_differences", ADJ, None),
    # prolongation (Sec. III.A)
    ("prolongation_parent_off_by_one",
     [("fine = parent.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)",
       "fine = np.roll(parent.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2), 1, "
       "axis=2)")],
     "test_prolongation_injection", {}, None),
    ("prolongation_without_neighbour_fill",
     [("parent = np.where(cfluid, sc, fill)", "parent = np.where(cfluid, sc, s_in)")],
     "test_prolongation_injection", {}, None),
    # Nernst model
    ("nernst_sigmoid_sign",
     [("        s_new[elec] = 1.0 / (1.0 + np.exp(-(kin.Vt - eta_t[elec])))",
       "        s_new[elec] = 1.0 / (1.0 + np.exp(-(kin.Vt + eta_t[elec])))")],
     "test_nernst_model_reaches_the_sbv_steady_state", dict(local_dt=True), 5.0),
    ("nernst_overpotential_sign",
     [("eta_i = 2.0 * np.arcsinh(-T[elec] / (2.0 * kappa[elec] * root))",
       "eta_i = 2.0 * np.arcsinh(T[elec] / (2.0 * kappa[elec] * root))")],
     "test_nernst_model_reaches_the_sbv_steady_state", dict(local_dt=True), 5.0),
]


def _load(edits, name):
    src = open(SOURCE_PATH).read()
    for old, new in edits:
        assert src.count(old) == 1, "planted edit of %s does not match once: %r" % (name, old)
        src = src.replace(old, new)
    mod = types.ModuleType("oracle_soc_" + name)
    sys.modules[mod.__name__] = mod       # dataclasses resolve annotations through it
    try:
        exec(compile(src, mod.__name__, "exec"), mod.__dict__)
    except BaseException:
        del sys.modules[mod.__name__]
        raise
    return mod


def _run_pin(monkeypatch, mod, pin, kwargs, limit):
    """Runs the named pin against module ``mod``; returns None if it passed, else the
    reason it failed."""
    monkeypatch.setattr(pins, "soc", mod)

    def alarm(signum, frame):
        raise PinTimeout()

    old = signal.signal(signal.SIGALRM, alarm) if limit else None
    if limit:
        signal.setitimer(signal.ITIMER_REAL, limit)
    try:
        getattr(pins, pin)(**kwargs)
        return None
    except AssertionError:
        return "assertion"
    except PinTimeout:
        return "did not finish in %.0f s" % limit
    except RuntimeError as e:           # the oracle's own non-convergence errors
        assert "oracle" in str(e), "planted edit broke the copy: %r" % e
        return "non-convergence"
    finally:
        if limit:
            signal.setitimer(signal.ITIMER_REAL, 0)
            signal.signal(signal.SIGALRM, old)


def test_unmodified_copy_passes_every_named_pin(monkeypatch):
    mod = _load([], "unmodified")
    try:
        seen = set()
        for _, _, pin, kwargs, _ in MUTATIONS:
            key = (pin, tuple(sorted(kwargs.items())))
            if key in seen:
                continue
            seen.add(key)
            assert _run_pin(monkeypatch, mod, pin, kwargs, None) is None, key
    finally:
        del sys.modules[mod.__name__]


@pytest.mark.parametrize("name,edits,pin,kwargs,limit", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_its_pin(monkeypatch, name, edits, pin, kwargs, limit):
    mod = _load(edits, name)
    try:
        import warnings
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            why = _run_pin(monkeypatch, mod, pin, kwargs, limit)
    finally:
        del sys.modules[mod.__name__]
    assert why is not None, "%s: %s still passes" % (name, pin)
