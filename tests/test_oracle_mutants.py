"""Planted mistakes: each plausible slip in the oracle (a dropped term, a
flipped sign, a transposed index, a garbled coefficient) is compiled into a
throw-away copy of the oracle, and at least one pin must fail on it. This
shows the pins constrain every part of the oracle."""
import os
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "kin_oracle.c")

MUTANTS = [
    ("reactant sign in omega", "if (m->reac[2 * j + s] >= 0) omega[m->reac[2 * j + s]] -= q;",
     "if (m->reac[2 * j + s] >= 0) omega[m->reac[2 * j + s]] += q;",
     [pins.test_unimolecular_decay_closed_form]),
    ("third-body factor dropped", "                q *= M;\n", "                q *= 1.0;\n",
     [pins.test_third_body_unit_efficiency_is_total_concentration]),
    ("density units", "rho = p * Wbar / (ORC_R * T) * 1e-6;", "rho = p * Wbar / (ORC_R * T) * 1e-3;",
     [pins.test_third_body_unit_efficiency_is_total_concentration,
      pins.test_quadratic_decay_closed_form_rate]),
    ("falloff blending inverted", "q *= Pr / (1.0 + Pr);", "q *= 1.0 / (1.0 + Pr);",
     [pins.test_falloff_limits]),
    ("Arrhenius sign", "exp(-m->Ea[j] / (ORC_R * T))", "exp(m->Ea[j] / (ORC_R * T))",
     [pins.test_unimolecular_decay_closed_form]),
    ("Butcher weight typo", "277.0 / 14336.0", "277.0 / 14363.0",
     [pins.test_rkck_table_is_the_printed_table, pins.test_rkck_order_conditions_from_oracle_table]),
    ("stage sum index", "acc += RK_B[st][l] * kk[l * n + i];", "acc += RK_B[st][l] * kk[st * n + i];",
     [pins.test_rkck_step_matches_printed_table_exactly]),
    ("RKCK growth exponent", "pow(errmax, -0.2)", "pow(errmax, -0.25)",
     [pins.test_rkck_controller_trace_on_linear_decay]),
    ("b_1 as printed (1/w0)", "    b[1] = b[2];\n", "    b[1] = 1.0 / w0;\n",
     [lambda: pins.test_rkc_first_stage_abscissa(8)]),
    ("RKC nu sign", "nu[j] = -b[j] / b[j - 2];", "nu[j] = b[j] / b[j - 2];",
     [lambda: pins.test_rkc_step_is_chebyshev_stability_polynomial(7)]),
    ("RKC gamma term dropped", "+ mut[j] * h * fj[i] + gt[j] * h * f0[i];", "+ mut[j] * h * fj[i];",
     [lambda: pins.test_rkc_step_is_chebyshev_stability_polynomial(7)]),
    ("damping kappa", "#define ORC_KAPPA (2.0 / 13.0)", "#define ORC_KAPPA (2.0 / 3.0)",
     [lambda: pins.test_rkc_first_stage_abscissa(8)]),
    ("error estimate weight", "0.4 * hh * (f0[i] + fx[i])", "0.5 * hh * (f0[i] + fx[i])",
     [pins.test_rkc_controller_trace_on_linear_decay]),
    ("PI controller exponent", "cbrt(err_prev) / pow(err, 2.0 / 3.0)", "cbrt(err_prev) / cbrt(err)",
     [pins.test_rkc_controller_trace_on_linear_decay]),
    ("stage rule constant", "sqrt(1.0 + 1.54 * h * sigma)", "sqrt(1.0 + 1.45 * h * sigma)",
     [pins.test_rkc_controller_trace_on_linear_decay]),
    ("Gershgorin column sums", "rowsum[i] += fabs((fx[i] - f0[i]) / eps);",
     "rowsum[k] += fabs((fx[i] - f0[i]) / eps);",
     [pins.test_gershgorin_on_linear_chain]),
    ("initial step factor", "0.1 * h0 / sqrt(e0)", "0.2 * h0 / sqrt(e0)",
     [pins.test_rkc_controller_trace_on_linear_decay]),
    ("power margin dropped", "    return 1.2 * sig;\n}", "    return 1.0 * sig;\n}",
     [pins.test_power_method_on_linear_chain]),
    ("power residual sign", "fz[i] -= f0[i];", "fz[i] += f0[i];",
     [pins.test_power_method_on_linear_chain, pins.test_power_method_diagonal_jacobian_exact]),
    ("power direction not renormalised", "for (i = 0; i < n; i++) v[i] = fz[i] * (dyn / wnorm);",
     "for (i = 0; i < n; i++) v[i] = fz[i];",
     [pins.test_power_method_on_linear_chain]),
    ("energy sign", "dydt[nS] = -hw / (rho * cpm);", "dydt[nS] = hw / (rho * cpm);",
     [pins.test_energy_f_conserves_mixture_enthalpy,
      lambda: pins.test_energy_adiabatic_temperature_rise_closed_form(oracle.RKCK)]),
    ("molar instead of mass heat capacity", "cpm += y[i] * m->cp[i] / m->W[i];",
     "cpm += y[i] * m->cp[i];",
     [pins.test_energy_f_conserves_mixture_enthalpy,
      lambda: pins.test_energy_adiabatic_temperature_rise_closed_form(oracle.RKCK)]),
    ("sensible enthalpy dropped", "hw += (m->Hf[i] + m->cp[i] * (T - ORC_TREF)) * omega[i];",
     "hw += m->Hf[i] * omega[i];",
     [pins.test_energy_f_conserves_mixture_enthalpy]),
    ("rates at a fixed temperature", "rho = production(m, T, p, k, k0, y, omega, C);",
     "rho = production(m, 1000.0, p, k, k0, y, omega, C);",
     [pins.test_energy_species_part_is_the_isothermal_f_at_the_state_temperature]),
    ("sigma refreshed every 20 steps", "if (since_sigma >= 25 || (last_rejected && !sigma_here)) {",
     "if (since_sigma >= 20 || (last_rejected && !sigma_here)) {",
     [lambda: pins.test_rkc_sigma_refresh_schedule(12.0, 1e-3)]),
    ("no sigma refresh after a rejection", "if (since_sigma >= 25 || (last_rejected && !sigma_here)) {",
     "if (since_sigma >= 25) {",
     [lambda: pins.test_rkc_sigma_refresh_schedule(12.0, 1e-3)]),
    ("sigma age never reset", "            since_sigma = 0;\n", "",
     [lambda: pins.test_rkc_sigma_refresh_schedule(12.0, 1e-3)]),
    ("sigma re-estimated at the point just estimated",
     "if (since_sigma >= 25 || (last_rejected && !sigma_here)) {",
     "if (since_sigma >= 25 || last_rejected) {",
     [lambda: pins.test_rkc_sigma_refresh_schedule(40.0, 1e-16)]),
    ("stage cap dropped",
     "            s = ORC_SMAX;\n            hh = ((ORC_SMAX - 1.0) * (ORC_SMAX - 1.0) - 1.0) / (1.54 * sigma);\n"
     "            last = 0;\n", "",
     [pins.test_rkc_stage_cap_on_stiff_linear_decay]),
    ("stage-cap step reset off by one", "hh = ((ORC_SMAX - 1.0) * (ORC_SMAX - 1.0) - 1.0) / (1.54 * sigma);",
     "hh = (ORC_SMAX * ORC_SMAX - 1.0) / (1.54 * sigma);",
     [pins.test_rkc_stage_cap_on_stiff_linear_decay]),
    ("RKCK minimum step", "double t = 0.0, h = dt, hmin = 1e-20 * dt;",
     "double t = 0.0, h = dt, hmin = 1e-22 * dt;",
     [pins.test_status_step_size_underflow]),
    ("RKC minimum step", "double t = 0.0, hmin = 1e-20 * dt, sigma,", "double t = 0.0, hmin = 1e-22 * dt, sigma,",
     [pins.test_status_step_size_underflow]),
]


@pytest.mark.parametrize("name,old,new,catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, catchers, monkeypatch):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor missing: " + name
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        lib = oracle.bind(oracle.compile_source(path, os.path.join(d, "libmutant.so")))
        monkeypatch.setattr(oracle, "_lib", lib)
        caught = 0
        for fn in catchers:
            try:
                fn()
            except AssertionError:
                caught += 1
        assert caught > 0, "no pin caught: " + name
