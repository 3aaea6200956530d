"""The oracle's pins catch plausible mistakes: each case plants one (a wrong constant, sign, exponent, index or a
dropped term) in a copy of oracle.c, builds that copy on its own, runs the pin that covers the code under it and
expects that pin to fail. The committed oracle is untouched; the same pins pass on it (test_oracle_pins.py)."""
import inspect
import os
import shutil
import subprocess

import pytest

import oracle as O
import test_oracle_mr as MR
import test_oracle_pins as P
import test_oracle_refined_pf as RP
from paper_1509_04953_gb300 import synth

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")
HDR = os.path.join(os.path.dirname(O.__file__), "oracle.h")


def _replace_once(old, new):
    def f(src):
        assert src.count(old) == 1, old
        return src.replace(old, new)
    return f


def _halve_basic_plastic_strain(src):
    # the basic scheme's state update (a7): the plastic strain takes half the converged shear rates
    anchor = "for (int I = 0; I < 6; ++I) tau += M[6 * a + I] * sigk[I * N3 + v];"
    line = "s->epsp[I * N3 + v] += dt * ep;"
    assert src.count(anchor) == 1
    j = src.index(line, src.index(anchor))
    return src[:j] + "s->epsp[I * N3 + v] += 0.5 * dt * ep;" + src[j + len(line):]


# (case, mutation, pin, pin arguments besides the material)
CASES = [
    ("green_operator_constant",        # Gamma0's second term with lam0 + mu0 for lam0 + 2 mu0
     _replace_once("double c2 = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0));",
                   "double c2 = (lam0 + mu0) / (mu0 * (lam0 + mu0));"),
     P.test_gamma0_projection_properties, {}),
    ("fft_twiddle_sign",
     _replace_once("cexp(sign * 2.0 * PI * IU * (double)k / (double)len)",
                   "cexp(-sign * 2.0 * PI * IU * (double)k / (double)len)"),
     P.test_fft_matches_brute_dft, dict(n=4)),
    ("km_square_root_dropped",         # k1 rho_F instead of k1 sqrt(rho_F)
     _replace_once("(p->k1 * srf - p->k2 * rho[a])", "(p->k1 * rf - p->k2 * rho[a])"),
     P.test_km_single_system_closed_form, dict(sense=1.0)),
    ("km_absolute_shear_dropped",      # (k1 sqrt(rho_F) - k2 rho) gdot instead of ... |gdot|
     _replace_once("rho[a] = rho[a] + dt * (p->k1 * srf - p->k2 * rho[a]) * fabs(gdot[a]);",
                   "rho[a] = rho[a] + dt * (p->k1 * srf - p->k2 * rho[a]) * gdot[a];"),
     P.test_km_single_system_closed_form, dict(sense=-1.0)),
    ("flow_rule_prefactor",            # the shear rate off by a factor its tangent and potential do not share
     _replace_once("gd = p->gdot0 * pw * (x < 0.0 ? -1.0 : 1.0);", "gd = 0.5 * p->gdot0 * pw * (x < 0.0 ? -1.0 : 1.0);"),
     P.test_newton_tangent_and_residual, {}),
    ("slip_direction_sign",            # [1 0 -1] on the (1 -1 1) plane written as [1 0 1]
     _replace_once("{{0, 1, 1}, {1, 0, -1}, {1, 1, 0}},", "{{0, 1, 1}, {1, 0, 1}, {1, 1, 0}},"),
     P.test_rotation_and_slip_geometry, {}),
    ("pf_gradient_coefficient",        # kappa = l/2 instead of 3l/4 in the phase-field step
     _replace_once("kap = 0.75 * l, gam = 1.5, Esc", "kap = 0.5 * l, gam = 1.5, Esc"),
     P.test_pf_flat_interface_tanh_profile_and_energy, {}),
    ("weibull_exponent",               # (-ln(1-u))^q instead of ^(1/q)
     _replace_once("return kc * pow(-log(1.0 - u), 1.0 / q);", "return kc * pow(-log(1.0 - u), q);"),
     P.test_weibull_sampler_matches_cdf, {}),
    ("sweep_softened_twice",
     _replace_once("if (gprev[v] < s->G && s->g[v] >= s->G) soften_voxel(s, v);",
                   "if (gprev[v] < s->G && s->g[v] >= s->G) { soften_voxel(s, v); soften_voxel(s, v); }"),
     P.test_pf_sweep_softening_and_recrystallised_fraction, {}),
    ("green_correction_sign",          # eps += Gamma0 : sigma instead of eps -= Gamma0 : sigma
     _replace_once("eh[I] = -a;", "eh[I] = a;"),
     P.test_elastic_laminate_closed_form, dict(scheme=0, ref_scale=1.0)),
    ("al_local_strain_sign",           # augmented Lagrangian, Sec. 2.1: e = C0^-1 (tau + sigma) for C0^-1 (tau - sigma)
     _replace_once("for (int J = 0; J < 6; ++J) st += S0[6 * I + J] * (tau[J] - sg[J]);",
                   "for (int J = 0; J < 6; ++J) st += S0[6 * I + J] * (tau[J] + sg[J]);"),
     P.test_elastic_laminate_closed_form, dict(scheme=1, ref_scale=1.0)),
    ("plastic_strain_update_halved",
     _halve_basic_plastic_strain,
     P.test_converged_increment_checks_hold_for_the_oracle, dict(n=16, G=8)),
    ("voronoi_tie_to_larger_index",    # reading C21 gives ties to the smaller seed index
     _replace_once("if (best < 0 || d2 < best) { best = d2; arg = g; }", "if (best < 0 || d2 <= best) { best = d2; arg = g; }"),
     P.test_voronoi_brute_force, {}),
    ("nucleation_eligibility_four_neighbours",   # reading C13: six face neighbours, not four
     _replace_once("        for (int d = 0; d < 6; ++d)\n            if (s->g[nbr(s->n, v, d)] != s->g[v]) gb = 1;",
                   "        for (int d = 0; d < 4; ++d)\n            if (s->g[nbr(s->n, v, d)] != s->g[v]) gb = 1;"),
     P.test_nucleation_eligibility_is_the_six_face_neighbours, {}),
    ("pf_argmax_tie_to_larger_id",     # reading C21
     _replace_once("(e == be && id < bi)", "(e == be && id > bi)"),
     P.test_pf_argmax_ties_go_to_the_smaller_id, {}),
    ("pf_keep_tie_to_larger_id",       # reading C11: the K largest, ties to the smaller id
     _replace_once("    if (x->e < y->e) return 1;\n    return (x->id > y->id) - (x->id < y->id);",
                   "    if (x->e < y->e) return 1;\n    return (x->id < y->id) - (x->id > y->id);"),
     P.test_pf_active_set_keeps_the_largest_ties_to_smaller_id_and_counts_overflow, {}),
    ("pf_overflow_not_counted",        # reading C11: overflow counted
     _replace_once("if (no > K) { ovf += 1; no = K; }", "if (no > K) { no = K; }"),
     P.test_pf_active_set_keeps_the_largest_ties_to_smaller_id_and_counts_overflow, {}),
    ("pf_drop_threshold_times_ten",    # reading C11: drop below 1e-5
     _replace_once("if (en >= s->p.eta_drop) {", "if (en >= 10.0 * s->p.eta_drop) {"),
     P.test_pf_drop_threshold, {}),
    ("adjoint_density_chain_factor",   # d sqrt(rho_F) / d rho taken as 1 / sqrt(rho_F), without the 1/2
     _replace_once("+ sum_lr_gd / (2.0 * srf);", "+ sum_lr_gd / srf;"),
     P.test_oracle_adjoint_gradient_matches_central_differences, {}),
    # the Ma-Roters law (Sec. 2.2)
    ("mr_flow_rule_offset_sign",       # sinh((|tau| + tp)/tcut) instead of sinh((|tau| - tp)/tcut), Eq. FlowRule
     _replace_once("const double x = (at - tp) / tcut;", "const double x = (at + tp) / tcut;"),
     MR.test_flow_rule_limits_derivative_and_potential, {}),
    ("mr_dipole_distance_constant",    # 8 pi instead of 16 pi in the dipole distance, Eq. SSDEvolution
     _replace_once("(16.0 * PI * (1.0 - p->poisson) * fabs(tau[a]))", "(8.0 * PI * (1.0 - p->poisson) * fabs(tau[a]))"),
     MR.test_ssd_terms_one_by_one, {}),
    ("mr_gnd_one_sided_difference_sign",   # backward one-sided difference with its sign flipped, Eq. GNDEvolution
     _replace_once("else if (sm[i]) grad[i] = (f[v] - f[nm[i]]) / leff;", "else if (sm[i]) grad[i] = (f[nm[i]] - f[v]) / leff;"),
     MR.test_gnd_stencil_exact_on_linear_fields, dict(axis=0)),
    ("mr_projection_table_swapped",    # GNDs projected with the forest table in place of its own (Eq. RhoForest)
     _replace_once("fabs(gs[b] * tab[144 + 12 * a + b])", "fabs(gs[b] * tab[12 * a + b])"),
     MR.test_projection_closed_forms, {}),
    ("mr_leff_update_inverted",        # l_eff (1 + xi eps) instead of l_eff (1 + eps / xi), Eq. L0evolution
     _replace_once("return leff * (1.0 + orc_vm_strain(E) / xi);", "return leff * (1.0 + orc_vm_strain(E) * xi);"),
     MR.test_von_mises_measures, {}),
    ("mr_gnd_total_sum_not_norm",      # |rs| + |re| instead of sqrt(rs^2 + re^2) (reading R7)
     _replace_once("s->gnd[i] += dt * sqrt(rs[i] * rs[i] + re[i] * re[i]);", "s->gnd[i] += dt * (fabs(rs[i]) + fabs(re[i]));"),
     MR.test_state_update_wires_the_gnd_and_ssd_laws, {}),
    ("mr_softening_reaches_ssd",       # reading R9 keeps rho_SSD at a nucleus
     _replace_once("            s->gnd[a * N3 + v] = f * s->gnd[a * N3 + v];\n",
                   "            s->gnd[a * N3 + v] = f * s->gnd[a * N3 + v];\n            s->rho[a * N3 + v] = f * s->rho[a * N3 + v];\n"),
     MR.test_nucleation_softens_gnd_and_keeps_ssd, {}),
    # the 2:1 phase-field grid (Sec. 2.4)
    ("refined_interpolation_weights",  # the odd child weighted 1/4, 3/4 instead of 3/4, 1/4
     _replace_once("else { idx[0] = i; idx[1] = (i + 1) % n; wt[0] = 0.75; wt[1] = 0.25; }",
                   "else { idx[0] = i; idx[1] = (i + 1) % n; wt[0] = 0.25; wt[1] = 0.75; }"),
     RP.test_interpolation_constant_mean_and_linear_fields, {}),
    ("refined_restriction_tie_to_larger_id",   # equal summed order parameters go to the smaller id
     _replace_once("(sum == bsum && id < best)", "(sum == bsum && id > best)"),
     RP.test_restriction_recovers_grains_and_takes_the_larger_sum, {}),
    ("refined_driving_force_spacing",  # E' at the mechanics spacing dx instead of the PF spacing dx / 2
     _replace_once("p->b * p->b * (p->dx / s->r) / p->omega_gb;", "p->b * p->b * p->dx / p->omega_gb;"),
     RP.test_refined_boundary_velocity_uses_the_pf_spacing, {}),
]


@pytest.mark.parametrize("case,mutate,pin,kw", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(tmp_path, case, mutate, pin, kw):
    src = mutate(open(SRC).read())
    (tmp_path / "oracle.c").write_text(src)
    shutil.copy(HDR, tmp_path / "oracle.h")
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                           str(tmp_path / "oracle.c"), "-lm"])
    args = dict(kw)
    params = inspect.signature(pin).parameters
    if "mat" in params:
        args["mat"] = synth.Material()
    if "mrmat" in params:
        args["mrmat"] = synth.ma_roters_material()
    with O.using(so):
        with pytest.raises(AssertionError):
            pin(**args)
