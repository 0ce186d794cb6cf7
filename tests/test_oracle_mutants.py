"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch every one of them (CPU only; the oracle itself is not modified)."""
import os
import subprocess

import pytest

import oracle
import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "tdse_oracle.c")

# (name, text in tdse_oracle.c, replacement, the pin expected to catch it)
MUTANTS = [
    ("coupling_sign", "c_scale(r * E * kappa(l), f_at(g, x, l - 1, j))",
     "c_scale(-r * E * kappa(l), f_at(g, x, l - 1, j))", P.check_symmetric),
    ("kappa_formula", "return RSQRT(ll / (4 * ll - 1));", "return RSQRT(ll / (4 * ll + 1));",
     P.check_coupling_blocks),
    ("stencil5_coefficient", "s = c_add(s, c_scale(16, f_at(g, x, l, j + 1)));",
     "s = c_add(s, c_scale(15, f_at(g, x, l, j + 1)));", P.check_stencil_polynomials),
    ("stencil3_coefficient", "s = c_add(s, c_scale(-2, f_at(g, x, l, j)));",
     "s = c_add(s, c_scale(-1.999, f_at(g, x, l, j)));", P.check_stencil_polynomials),
    ("centrifugal", "(REAL)l * (REAL)(l + 1) / (2 * r * r)", "(REAL)l * (REAL)l / (2 * r * r)",
     P.check_hydrogen_convergence),
    ("coulomb_sign", "return -(REAL)g->Z / grid_r(g, j);", "return (REAL)g->Z / grid_r(g, j);",
     P.check_hydrogen_paper_values),
    ("odd_ghost_always", "if (g->ghost == 1 && j == -1)", "if (j == -1)",
     P.check_hydrogen_paper_values),
    ("taylor_printed_factor", "const REAL s = dt / (REAL)p;",
     "const REAL s = dt / (REAL)(p > 1 ? p - 1 : 1);", P.check_field_free_eigenstate),
    ("rk4_weights", "static const REAL b[4] = {1, 2, 2, 1};",
     "static const REAL b[4] = {2, 1, 2, 1};", P.check_field_free_eigenstate),
    ("rk4_stage_time", "(REAL)coupling(pulse, tn + dt)};", "(REAL)coupling(pulse, tn + 0.5 * dt)};",
     P.check_time_order),
    ("taylor_field_time", "taylor_step(g, (REAL)coupling(pulse, tn + 0.5 * dt)",
     "taylor_step(g, (REAL)coupling(pulse, tn)", P.check_time_order),
    ("lanczos_drop_beta", "w[i] = c_sub(w[i], c_scale(beta[j - 1], qprev[i]));",
     "w[i] = w[i];", P.check_dense_expm),
    ("lanczos_alpha_sign", "a += qj[i].re * w[i].re + qj[i].im * w[i].im;",
     "a += qj[i].re * w[i].re - qj[i].im * w[i].im;", P.check_dense_expm),
    ("lanczos_norm_rescale", "psi[i] = c_scale(nrm, s);", "psi[i] = s;",
     P.check_field_free_eigenstate),
    ("dipole_factor", "dip += 2 * kappa(l + 1) * h * s;", "dip += kappa(l + 1) * h * s;",
     P.check_observables),
    ("p_ground_conjugate", "-(REAL)ref0[2 * (j - 1) + 1]", "(REAL)ref0[2 * (j - 1) + 1]",
     P.check_observables),
    ("norm_weight", "out[0] = (double)(h * norm);", "out[0] = (double)(norm);",
     P.check_observables),
    ("yield_radius", "if (grid_r(g, j) <= (REAL)r_b) inside += a;", "inside += a;",
     P.check_norm_and_yield),
    ("mask_exponent", "pow(cos(x), 0.125)", "pow(cos(x), 0.25)", P.check_mask),
    ("envelope_period", "sin(M_PI * t / T);", "sin(2.0 * M_PI * t / T);", P.check_pulse),
    ("imag_energy_printed_factor", "e = -RLOG(n1 / n0) / (2 * (REAL)dt);", "e = -RLOG(n1 / n0) / ((REAL)dt);",
     P.check_imaginary_time_eigenstate),
    ("imag_lanczos_exponent_sign", "c_make(REXP(ph), 0)", "c_make(REXP(-ph), 0)",
     P.check_imaginary_time_ground_state),
    ("imag_taylor_sign", "term[i] = imag ? c_scale(-s, tmp[i])", "term[i] = imag ? c_scale(s, tmp[i])",
     P.check_imaginary_time_eigenstate),
    ("velocity_printed_signs", "w = c_add(w, c_scale(kappa(l), c_sub(d1_at(g, x, l - 1, j),",
     "w = c_add(w, c_scale(kappa(l), c_add(d1_at(g, x, l - 1, j),", P.check_velocity_gauge_operator),
    ("velocity_missing_c", "c_scale(E / (REAL)ORC_C_AU, w)", "c_scale(E, w)", P.check_velocity_gauge_operator),
    ("vecpot_sign", "return -ORC_C_AU * s;", "return ORC_C_AU * s;", P.check_vector_potential),
    ("first_derivative_weight", "s = c_add(s, c_scale(8, f_at(g, x, l, j + 1)));",
     "s = c_add(s, c_scale(7, f_at(g, x, l, j + 1)));", P.check_velocity_gauge_operator),
    ("rkf_stage_coefficient", "{1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197}",
     "{1932.0 / 2197, -7200.0 / 2197, 7269.0 / 2197}", P.check_rk_orders),
    ("cash_karp_node", "{0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1, 7.0 / 8}",
     "{0, 1.0 / 5, 3.0 / 10, 3.0 / 5, 1, 5.0 / 8}", P.check_rk_orders),
    ("cash_karp_lower_weight", "277.0 / 14336, 1.0 / 4}", "277.0 / 14336, 1.0 / 2}", P.check_rk_orders),
    ("dormand_prince_lower_weight", "-92097.0 / 339200, 187.0 / 2100, 1.0 / 40}",
     "-92097.0 / 339200, 187.0 / 2100, 1.0 / 4}", P.check_rk_dormand_prince_step),
    ("merson_weights", "{1.0 / 6, 0, 0, 2.0 / 3, 1.0 / 6}", "{1.0 / 6, 0, 2.0 / 3, 0, 1.0 / 6}",
     P.check_rk_orders),
    ("rk_stage_time", "coupling(pulse, tn + tb->c[i] * dt)", "coupling(pulse, tn)", P.check_rk_orders),
    ("rk_keeps_lower_solution", "hi = c_add(hi, c_scale((REAL)dt * (REAL)tb->b2[i], ki));",
     "hi = c_add(hi, c_scale((REAL)dt * (REAL)tb->b1[i], ki));", P.check_rk_orders),
    ("sigma_counts_reals", "sig += RSQRT(d2 / (REAL)n);", "sig += RSQRT(d2 / (REAL)(2 * n));",
     P.check_rk_dormand_prince_step),
    ("sigma_no_sqrt", "sig += RSQRT(d2 / (REAL)n);", "sig += d2 / (REAL)n;", P.check_rk_orders),
    ("dipole_velocity_printed_factor", "pz += 2 * kappa(l + 1) * h * sp;", "pz += kappa(l + 1) * h * sp;",
     P.check_dipole_ehrenfest),
    ("dipole_velocity_centrifugal", "c_scale((REAL)(l + 1) / r, a));", "c_scale((REAL)l / r, a));",
     P.check_dipole_ehrenfest),
    ("dipole_velocity_gauge_term", "(REAL)orc_vecpot(pulse, t) / (REAL)ORC_C_AU * norm",
     "-(REAL)orc_vecpot(pulse, t) / (REAL)ORC_C_AU * norm", P.check_dipole_ehrenfest),
    ("dipole_accel_field_sign", "(double)(-(REAL)orc_field(pulse, t) * norm", "(double)((REAL)orc_field(pulse, t) * norm",
     P.check_dipole_ehrenfest),
    ("dipole_accel_power", "sf += re / (r * r);", "sf += re / r;", P.check_dipole_ehrenfest),
    ("flux_printed_sign", "tot += fb[l].re * db[l].im - fb[l].im * db[l].re;",
     "tot -= fb[l].re * db[l].im - fb[l].im * db[l].re;", P.check_flux_continuity),
    ("flux_gauge_term_factor", "tot += 2 * ac * kappa(l + 1)", "tot += ac * kappa(l + 1)",
     P.check_flux_angular_integral),
    ("harmonic_normalisation", "RSQRT((REAL)(2 * l + 1) / (4 * (REAL)M_PI))", "RSQRT((REAL)(2 * l + 1) / (2 * (REAL)M_PI))",
     P.check_flux_closed_form),
    ("legendre_recurrence", "((REAL)(2 * l + 1) * x * pl - (REAL)l * pm)", "((REAL)(2 * l + 1) * x * pl - (REAL)(l + 1) * pm)",
     P.check_flux_closed_form),
    ("flux_radius_off_by_one", "return best;", "return best + 1;", P.check_flux_continuity),
    ("sinea_missing_envelope_term", "+ 2.0 * W * cos(M_PI * t / T) * sin(ph)", "+ 0.0 * W * cos(M_PI * t / T) * sin(ph)",
     P.check_sinea_pulse),
    ("sinea_envelope_frequency", "const double W = M_PI / T,", "const double W = 2.0 * M_PI / T,",
     P.check_sinea_pulse),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, check):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"libmut_{name}.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", str(so), str(path), "-lm"], check=True)
    key = f"mutant-{name}"
    oracle.register_library(key, str(so))
    with pytest.raises(AssertionError):
        check(key)
