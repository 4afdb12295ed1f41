"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of an
oracle module (a dropped term, a flipped sign, a transposed operand, a wrong factor, an
index or time-sampling slip), swaps the mutated functions in for the duration of the test
and requires each of the named pins of ``test_oracle_pins`` to fail (every mutant is
caught by at least one pin; the lists name the pins that catch it).

Everything runs on the CPU against the FP64 oracle; the CUDA library is not involved.
"""
import inspect

import pytest

import oracle.adjoint
import oracle.demag
import oracle.llg
import oracle.newell
import test_oracle_pins as P

MODULES = {"newell": oracle.newell, "demag": oracle.demag, "llg": oracle.llg,
           "adjoint": oracle.adjoint}
# every function and class each module (and the pins) holds, as imported
ORIGINAL = {(m.__name__, k): v for m in list(MODULES.values()) + [P] for k, v in vars(m).items()
            if inspect.isfunction(v) or inspect.isclass(v)}

PINS = {
    "cube": P.test_cube_self_term_is_one_third,
    "aharoni": lambda: P.test_self_term_matches_aharoni_and_has_unit_trace((1e-9, 2e-9, 3e-9)),
    "body_avg": lambda: P.test_body_average_equals_prism_factor(
        (64, 8, 2), (3.90625e-9, 3.90625e-9, 3e-9)),
    "quad_near": lambda: P.test_tensor_matches_dipole_quadrature((2, 1, 1)),
    "quad_far": lambda: P.test_tensor_matches_dipole_quadrature((30, 7, 2)),
    "asym_order": P.test_far_field_asymptote_converges_at_fourth_order,
    "symmetry": P.test_tensor_symmetries,
    "fft_direct": lambda: P.test_fft_convolution_equals_direct_sum((5, 3, 2)),
    "far_direct": P.test_direct_sum_far_branch_equals_fft,
    "single_cell": P.test_single_cell_field_is_minus_self_tensor_times_m,
    "self_adjoint": P.test_demag_is_self_adjoint_and_energy_positive,
    "cosine": lambda: P.test_neumann_cosine_mode_is_eigenvector(2),
    "gradient": P.test_field_is_minus_energy_gradient,
    "unit": P.test_llg_torque_is_orthogonal_and_step_keeps_unit_length,
    "macrospin": P.test_macrospin_closed_form_first_order,
    "heun": P.test_heun_macrospin_second_order,
    "pulse_euler": lambda: P.test_pulsed_field_macrospin_euler(1.6e-11),
    "pulse_heun": lambda: P.test_pulsed_field_macrospin_heun_second_order(1.6e-11),
    "step_start": P.test_euler_samples_field_at_step_start,
    "pulse_off": P.test_pulse_off_leaves_macrospin_still,
    "kittel": P.test_kittel_frequency_of_flat_cell,
    "damping": P.test_energy_decreases_under_damping,
    "adj_fd": P.test_adjoint_matches_central_differences,
    "adj_dot": P.test_adjoint_step_dot_product,
}

# (id, module, exact source text, its mutated form, pins expected to catch it)
MUTANTS = [
    # cell-averaged tensor
    ("f_arctan_sign", "newell", "t = t - x * y * z * np.arctan(", "t = t + x * y * z * np.arctan(",
     ["cube", "aharoni"]),
    ("f_last_term_dropped", "newell", "t = t + (2.0 * x2 - y2 - z2) * R / 6.0", "t = t",
     ["aharoni", "body_avg", "quad_near"]),
    ("g_last_term_sign", "newell", "t = t - x * y * R / 3.0", "t = t + x * y * R / 3.0",
     ["quad_near"]),
    ("second_difference_weights", "newell", "_W = {-1: -1.0, 0: 2.0, 1: -1.0}",
     "_W = {-1: 1.0, 0: 2.0, 1: 1.0}", ["cube", "aharoni"]),
    ("yz_from_xz_arguments", "newell", "nyz = _second_difference(newell_g, Y, Z, X, dy, dz, dx)",
     "nyz = _second_difference(newell_g, X, Z, Y, dx, dz, dy)", ["quad_near", "symmetry"]),
    ("asymptote_correction_dropped", "newell", "out.append(dip - pref * corr / 12.0)",
     "out.append(dip)", ["asym_order", "quad_far"]),
    ("asymptote_correction_sign", "newell", "out.append(dip - pref * corr / 12.0)",
     "out.append(dip + pref * corr / 12.0)", ["asym_order", "quad_far"]),
    ("dipole_sign", "newell", "dip = pref * (dab * r2 - 3.0 * x[a] * x[b]) / r5",
     "dip = pref * (3.0 * x[a] * x[b] - dab * r2) / r5", ["quad_far", "body_avg"]),
    ("newell_region_too_small", "newell", "near = cheb <= r_switch", "near = cheb <= r_switch - 20",
     ["body_avg"]),
    # demag convolution
    ("padding_too_short", "demag", "while p < 2 * n - 1:", "while p < n:", ["fft_direct"]),
    ("transposed_operand_in_Hy", "demag", "sxy * Mh[0] + syy * Mh[1] + syz * Mh[2]",
     "sxy * Mh[0] + syy * Mh[1] + sxz * Mh[2]", ["fft_direct", "self_adjoint"]),
    ("convolution_sign", "demag", "np.stack([-np.fft.irfftn(", "np.stack([np.fft.irfftn(",
     ["fft_direct", "single_cell", "self_adjoint"]),
    ("correlation_instead_of_convolution_in_z", "demag", "iz = np.arange(-(nz - 1), nz) % P[0]",
     "iz = np.arange(nz - 1, -nz, -1) % P[0]", ["fft_direct"]),
    # exchange, anisotropy, Zeeman and the energies
    ("laplacian_back_bond_sign", "llg", "out[tuple(hi)] -= d", "out[tuple(hi)] += d",
     ["cosine", "gradient"]),
    ("laplacian_cell_sizes_swapped", "llg",
     "for axis, h in ((3, cell[0]), (2, cell[1]), (1, cell[2])):\n        if m.shape[axis] < 2:",
     "for axis, h in ((3, cell[2]), (2, cell[1]), (1, cell[0])):\n        if m.shape[axis] < 2:",
     ["gradient"]),
    ("exchange_factor_two_dropped", "llg", "return 2.0 * p.A / (MU0 *", "return p.A / (MU0 *",
     ["gradient"]),
    ("anisotropy_on_z", "llg", "h[0] = 2.0 * p.Ku / (MU0 * np.asarray(p.Ms, dtype=np.float64)) * m[0]",
     "h[2] = 2.0 * p.Ku / (MU0 * np.asarray(p.Ms, dtype=np.float64)) * m[2]",
     ["gradient", "kittel"]),
    ("anisotropy_sign", "llg", "h[0] = 2.0 * p.Ku", "h[0] = -2.0 * p.Ku", ["gradient", "kittel"]),
    ("zeeman_ignores_envelope", "llg", "h = field_scale(t, p.pulse) * np.asarray(p.hext",
     "h = np.asarray(p.hext", ["pulse_off", "pulse_euler"]),
    ("demag_energy_half_dropped", "llg", "e_d = -0.5 * MU0 * V", "e_d = -MU0 * V", ["gradient"]),
    ("zeeman_energy_halved", "llg", "e_z = -MU0 * V", "e_z = -0.5 * MU0 * V", ["gradient"]),
    ("anisotropy_energy_sign", "llg", "np.sum(1.0 - m[0] ** 2)", "np.sum(m[0] ** 2)", ["gradient"]),
    # LLG right-hand side and the integrators
    ("damping_sign", "llg", "(mxh + alpha * np.cross(m, mxh, axis=0))",
     "(mxh - alpha * np.cross(m, mxh, axis=0))", ["damping", "macrospin"]),
    ("precession_sign", "llg", "(mxh + alpha * np.cross(m, mxh, axis=0))",
     "(-mxh + alpha * np.cross(m, mxh, axis=0))", ["macrospin"]),
    ("gilbert_factor_dropped", "llg", "-gamma0 / (1.0 + alpha * alpha) *", "-gamma0 *",
     ["macrospin"]),
    ("euler_not_renormalised", "llg",
     "return normalise(m + dt * llg_rhs(m, heff(m, p, demag, t=t), p.alpha, p.gamma0))",
     "return m + dt * llg_rhs(m, heff(m, p, demag, t=t), p.alpha, p.gamma0)", ["unit"]),
    ("euler_field_at_step_end", "llg",
     "return normalise(m + dt * llg_rhs(m, heff(m, p, demag, t=t), p.alpha, p.gamma0))",
     "return normalise(m + dt * llg_rhs(m, heff(m, p, demag, t=t + dt), p.alpha, p.gamma0))",
     ["step_start"]),
    ("heun_corrector_only_k2", "llg", "m + 0.5 * dt * (k1 + k2)", "m + dt * k2", ["heun"]),
    ("heun_corrector_field_at_t_n", "llg", "heff(ms, p, demag, t=t + dt)", "heff(ms, p, demag, t=t)",
     ["pulse_heun"]),
    ("time_not_advanced", "llg", "        t = t + dt\n", "        t = t\n", ["pulse_euler"]),
    ("ramp_reversed", "llg", "return (t2 - t) / (t2 - t1)", "return (t - t1) / (t2 - t1)",
     ["pulse_euler", "pulse_heun"]),
    ("switch_on_edge_exclusive", "llg", "if t < t0:", "if t <= t0:", ["step_start", "pulse_heun"]),
    # discrete adjoint
    ("adjoint_projection_dropped", "adjoint",
     "mu = (lam_next - m1 * (m1 * lam_next).sum(axis=0, keepdims=True)) / un",
     "mu = lam_next / un", ["adj_dot"]),
    ("adjoint_damping_sign", "adjoint", "nu = dt * c * (cr(m, mu) - p.alpha", "nu = dt * c * (cr(m, mu) + p.alpha",
     ["adj_dot", "adj_fd"]),
    ("adjoint_demag_without_Ms", "adjoint", "lam = lam + Ms * d_nu", "lam = lam + d_nu", ["adj_dot"]),
    ("adjoint_exchange_transposed", "adjoint", "laplacian(2.0 * p.A / (MU0 * Ms) * nu, p.cell)",
     "2.0 * p.A / (MU0 * Ms) * laplacian(nu, p.cell)", ["adj_dot"]),
    ("adjoint_anisotropy_component", "adjoint", "lam[0] = lam[0] + 2.0 * p.Ku / (MU0 * Ms) * nu[0]",
     "lam[0] = lam[0] + 2.0 * p.Ku / (MU0 * Ms) * nu[2]", ["adj_dot"]),
    ("adjoint_ms_gradient_sign", "adjoint", "g_ms = (m * d_nu).sum(axis=0) - (nu * h_loc)",
     "g_ms = (m * d_nu).sum(axis=0) + (nu * h_loc)", ["adj_fd"]),
    ("adjoint_steps_in_forward_order", "adjoint", "for n in range(steps - 1, -1, -1):",
     "for n in range(steps):", ["adj_fd"]),
]


def _plant(monkeypatch, module, old, new):
    """Execute a copy of ``module`` with ``old`` replaced by ``new`` and swap every function or
    class it defines into each module that holds the original object under the same name."""
    src = inspect.getsource(module)
    assert src.count(old) == 1, f"mutation site not unique in {module.__name__}: {old!r}"
    ns = {"__name__": module.__name__, "__package__": module.__package__,
          "__file__": module.__file__}
    exec(compile(src.replace(old, new), module.__file__, "exec"), ns)
    holders = list(MODULES.values()) + [P]
    swapped = 0
    for name, obj in vars(module).items():
        if not (inspect.isfunction(obj) or inspect.isclass(obj)) or name not in ns:
            continue
        if getattr(obj, "__module__", None) != module.__name__:
            continue
        for h in holders:
            if getattr(h, name, None) is obj:
                monkeypatch.setattr(h, name, ns[name])
                swapped += 1
    assert swapped > 0


@pytest.mark.parametrize("mid,mod,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(monkeypatch, mid, mod, old, new, pins):
    _plant(monkeypatch, MODULES[mod], old, new)
    passed = []
    for name in pins:
        try:
            PINS[name]()
            passed.append(name)
        except AssertionError:
            pass
    assert not passed, f"planted mistake {mid} passed the pins {passed}"


def test_unmutated_pins_pass():
    """The same pin calls pass on the unmodified oracle (so a catch above is the mistake's)."""
    for name, pin in PINS.items():
        pin()


def test_mutants_leave_the_oracle_untouched():
    """Each mutant is undone after its test: every module again holds its original objects."""
    for m in list(MODULES.values()) + [P]:
        for k, v in vars(m).items():
            if (m.__name__, k) in ORIGINAL:
                assert v is ORIGINAL[(m.__name__, k)], (m.__name__, k)
