"""The oracle pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, an index off by
one, a transposed coefficient) in a private copy of the oracle's C source,
builds it on the CPU, swaps it in, and checks that the named pin now fails.
"""
import os
import subprocess

import pytest

import oracle as O
import oracle.oracle as OO
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(OO.__file__), "fwi_oracle.c")

MUTANTS = [
    # (id, original text, planted text, pin that must fail)
    ("adjoint_drops_sponge_in_lambda2", "(1.0 - gam[j] * dt) / (1.0 + gam[j] * dt) * l2[j]", "l2[j]",
     lambda: P.test_tangent_linear_adjoint_dot(2)),
    ("adjoint_wrong_operand_in_laplacian", "t[j] = c / (1.0 + gam[j] * dt) * l1[j];", "t[j] = c * l1[j];",
     lambda: P.test_tangent_linear_adjoint_dot(2)),
    ("stencil_coefficient_typo", "8.0 / 315.0", "8.0 / 305.0",
     lambda: P.test_lap8_exact_on_degree9_polynomials(2)),
    ("records_previous_time_level", "d[(long)n * nrec + r] = pn[rec_idx[r]];", "d[(long)n * nrec + r] = p[rec_idx[r]];",
     P.test_forward_2d_matches_green_function),
    ("gradient_pairs_wrong_snapshot", "or_lap8(g, snaps + (long)(k - 1) * np, Lp);",
     "or_lap8(g, snaps + (long)(k < g->nt ? k : k - 1) * np, Lp);",
     lambda: P.test_gradient_matches_central_differences(2)),
    ("fold_drops_chain_rule_factor", "gv[k] += 2.0 * v[k]", "gv[k] += v[k]",
     lambda: P.test_gradient_matches_central_differences(2)),
    ("renoise_uses_abar_t_in_x0_weight", "double c0 = sqrt(abar_prev) * beta_t", "double c0 = sqrt(abar_t) * beta_t",
     P.test_renoise_preserves_ddpm_marginal),
    ("langevin_ascends", "z[i] - eta * grad[i]", "z[i] + eta * grad[i]",
     P.test_langevin_ula_stationary_variance),
    ("precond_noise_not_matched", "nu * sqrt(G) * or_gauss", "nu * or_gauss",
     P.test_precond_langevin_matched_noise_stationary_variance),
    ("precond_rms_of_first_sample_only", "double r = sqrt(msum / (double)per);",
     "static double r0; double r = s == 0 ? (r0 = sqrt(msum / (double)per)) : r0;",
     P.test_precond_langevin_closed_form_steps_and_per_sample_scale),
    ("precond_no_bias_correction", "double cv = k > 0 ? 1.0 - pow(alpha, (double)k) : 1.0;", "double cv = 1.0;",
     P.test_precond_langevin_closed_form_steps_and_per_sample_scale),
    ("shuffle_off_by_one", "(unsigned __int128)(i + 1)) >> 64", "(unsigned __int128)(i)) >> 64",
     P.test_fisher_yates_uniform_chi2),
    ("sponge_sign_flipped", "pn[k] = (2.0 * p[k] - (1.0 - gam[k] * dt) * pm[k]", "pn[k] = (2.0 * p[k] - (1.0 + gam[k] * dt) * pm[k]",
     P.test_sponge_absorbs_reflections),
]


@pytest.mark.parametrize("mid,orig,planted,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, mid, orig, planted, pin):
    src = open(SRC).read()
    assert src.count(orig) == 1, "mutation anchor not found exactly once"
    c = tmp_path / "mutant.c"
    c.write_text(src.replace(orig, planted))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    saved = O.lib()
    OO._lib = OO.load(str(so))
    try:
        with pytest.raises((AssertionError, MemoryError, ValueError, FloatingPointError)):
            with __import__("numpy").errstate(all="ignore"):
                pin()
    finally:
        OO._lib = saved
