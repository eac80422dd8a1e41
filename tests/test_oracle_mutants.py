"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that
at least one pin of test_oracle_pins.py fails for each.  This is what makes
the pins trustworthy: they are not satisfied by a wrong oracle."""
from __future__ import annotations

import pytest

import test_oracle_pins as pins
from oracle import pf_oracle

MUTANTS = {
    # name: (original text, replacement, pin that must fail)
    "drop_gaussian_normaliser": ("inc = inc - lognorm;", "inc = inc;", "c_zero"),
    "drop_log_N": ("inc = inc - log((double)N);", "inc = inc;", "c_zero"),
    "weight_sign": ("e[i] = -0.5 * acc;", "e[i] = 0.5 * acc;", "c_zero"),
    "transpose_C": ("mu = mu + Cm[p * U + u] *", "mu = mu + Cm[u * P + p] *", "single_particle"),
    "power_law_propensity": ("return x * (x - 1) / 2; /* p == 2 */", "return x * x;",
                             "second_order"),
    "time_times_a0": ("double tau = E / a0;", "double tau = E * a0;", "birth_death_law"),
    "ziggurat_no_wedge_test": ("if (y < exp(-x)) return x;", "return x;", "exp_law"),
    "ziggurat_tail_without_offset": ("return zig_r + -log(u1);", "return -log(u1);", "exp_law"),
    "ziggurat_layer_bits": ("int i = (int)(W & 0x7FF);", "int i = (int)(W & 0x3FF);", "exp_law"),
    "stoichiometry_sign": ("x[u] += net->prod[chosen * net->U + u] - net->reac[chosen * net->U + u];",
                           "x[u] += net->reac[chosen * net->U + u] - net->prod[chosen * net->U + u];",
                           "birth_death_law"),
    "selection_no_prefix": ("if (target < S[r]) { chosen = r; break; }",
                            "if (target < a[r]) { chosen = r; break; }", "ge_moments"),
    "resample_non_strict": ("while (!((uint64_t)N * Q[i] > point)) i++;",
                            "while (!((uint64_t)N * Q[i] >= point)) i++;", "resampling"),
    "resample_no_offset": ("uint64_t point = u + (uint64_t)j * W;",
                           "uint64_t point = (uint64_t)j * W;", "resampling"),
    "philox_key_bump": ("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE84u;", "philox"),
    "weights_before_resample_ignored": ("q[i] = (uint64_t)ldexp(exp(e[i] - emax), 32);",
                                        "q[i] = (uint64_t)1 << 32;", "unbiased"),
    "initial_span_short": ("uint64_t span = (uint64_t)((int64_t)mdl->x0_hi[u] - x0[u] + 1);",
                           "uint64_t span = (uint64_t)((int64_t)mdl->x0_hi[u] - x0[u]);",
                           "init_uniform"),
    "initial_same_word": ("v += (int64_t)(((uint64_t)w[u & 3] * span) >> 32);",
                          "v += (int64_t)(((uint64_t)w[0] * span) >> 32);", "init_uniform"),
    "state_variance_ignored": ("v = v + mdl->obs_var[p * U + u] * (double)x[(size_t)i * U + u];",
                               "v = v;", "model_unbiased"),
    "state_variance_log_dropped": ("lv = lv + log(v);", "lv = lv;", "model_unbiased"),
    "composed_rate_transposed": ("v = v + net->rate_coef[r * net->d + c] * theta[c];",
                                 "v = v + net->rate_coef[c * net->R + r] * theta[c];",
                                 "model_unbiased"),
    "grid20_truncates": ("ldexp(nearbyint(ldexp(e, 20)), -20)", "ldexp(trunc(ldexp(e, 20)), -20)",
                         "grid20"),
    "grid20_width": ("ldexp(nearbyint(ldexp(e, 20)), -20)", "ldexp(nearbyint(ldexp(e, 19)), -19)",
                     "grid20"),
    "grid20_max_not_rounded": ("exp(grid20(e[i]) - grid20(emax))", "exp(grid20(e[i]) - emax)",
                               "quantise"),
    "grid20_dropped": ("exp(grid20(e[i]) - grid20(emax))", "exp(e[i] - emax)", "quantise"),
}

CHECKS = {
    "c_zero": lambda o, kat: pins.check_weights_c_zero(o),
    "single_particle": lambda o, kat: pins.check_single_particle(o),
    "second_order": lambda o, kat: pins.check_second_order_convention(o, n=4000),
    "birth_death_law": lambda o, kat: pins.check_birth_death_law(o, n=4000),
    "ge_moments": lambda o, kat: pins.check_gene_expression_moments(o, n=4000),
    "resampling": lambda o, kat: pins.check_resampling(o),
    "philox": lambda o, kat: pins.check_philox(o, kat),
    "unbiased": lambda o, kat: pins.check_unbiased(o, S=150, N=100),
    "exp_law": lambda o, kat: pins.check_exp_variates(o),
    "init_uniform": lambda o, kat: pins.check_initial_uniform(o),
    "model_unbiased": lambda o, kat: pins.check_model_unbiased(o, S=150, N=100),
    "grid20": lambda o, kat: pins.check_grid20(o),
    "quantise": lambda o, kat: pins.check_quantised_weights(o),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_detects_mutant(name, tmp_path, kat_vectors):
    old, new, check = MUTANTS[name]
    src = pf_oracle.source_text()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    variant = pf_oracle.compile_variant(src.replace(old, new), tmp_path)
    with pytest.raises(AssertionError):
        CHECKS[check](variant, kat_vectors)


def test_unmutated_copy_passes_all_checks(tmp_path, kat_vectors):
    """The same harness on an unmodified copy: every check passes."""
    variant = pf_oracle.compile_variant(pf_oracle.source_text(), tmp_path)
    for check in CHECKS.values():
        check(variant, kat_vectors)
