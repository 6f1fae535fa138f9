"""Each pin set must catch plausible mistakes in the oracle.

A mutant is a copy of oracle.c with one deliberate mistake (a dropped term,
a wrong sign, a wrong index, a transposed operand), compiled on the CPU into a
temporary directory.  Running every pin against it must fail at least once.
"""
import os
import tempfile

import pytest

import oracle
from oracle_checks import ALL_CHECKS

MUTANTS = {
    "csr_wrong_gather_index": ("s += val[k] * x[idx[k]];", "s += val[k] * x[i];"),
    "csr_dropped_value": ("s += val[k] * x[idx[k]];", "s += x[idx[k]];"),
    "sym_dropped_transpose": ("if (j > i) y[j] += val[k] * x[i];", "(void)0;"),
    "sym_transpose_wrong_operand": ("if (j > i) y[j] += val[k] * x[i];", "if (j > i) y[j] += val[k] * x[j];"),
    "sym_diagonal_twice": ("if (j > i) y[j] += val[k] * x[i];", "if (j >= i) y[j] += val[k] * x[i];"),
    "csc_transposed": ("y[rowidx[k]] += val[k] * x[j];", "y[j] += val[k] * x[rowidx[k]];"),
    "cg_x_sign": ("x[i] += alpha * p[i];   /* x += alpha p */", "x[i] -= alpha * p[i];"),
    "cg_r_uses_p": ("r[i] -= alpha * q[i];   /* r -= alpha A p */", "r[i] -= alpha * p[i];"),
    "cg_alpha_inverted": ("double alpha = rr / pq;", "double alpha = pq / rr;"),
    "cg_beta_inverted": ("double beta = rr_new / rr;", "double beta = rr / rr_new;"),
    "cg_beta_dropped": ("p[i] = r[i] + beta * p[i];  /* p = r + beta p */", "p[i] = r[i];"),
    "cg_initial_residual_sign": ("r[i] = b[i] - q[i];\n#pragma omp parallel for schedule(static)\n  for",
                                 "r[i] = b[i] + q[i];\n#pragma omp parallel for schedule(static)\n  for"),
    "cg_no_true_residual_confirm": ("if (info->rel_res_true <= tol) break;", "break;"),
    "dot_long_drops_term": ("s += (long double)a[i] * (long double)b[i];",
                            "if (i) s += (long double)a[i] * (long double)b[i];"),
    "f32_beta_dropped": ("p[i] = r[i] + beta * p[i];\n  }\n  free(r);", "p[i] = r[i];\n  }\n  free(r);"),
    "ir_missing_scale": ("x[i] += nr * (double)d[i];", "x[i] += (double)d[i];"),
    "ir_residual_sign": ("r[i] = b[i] - r[i];", "r[i] = r[i] - b[i];"),
    "abs_spmv_signed": ("double a = fabs(val[k]);", "double a = val[k];"),
    "f32_dot_left_to_right": ("  if (n <= 8) {\n    float s", "  if (1) {\n    float s"),
    "f32_dot_wrong_half": ("dot_f(n - h, a + h, b + h)", "dot_f(n - h, a + h, b)"),
    "grad_sym_drops_transpose": ("g[k] = -(lambda[r] * x[c] + lambda[c] * x[r]);", "g[k] = -(lambda[r] * x[c]);"),
    "grad_sym_doubles_diagonal": ("fmt == ORC_SYM_UPPER && c != r", "fmt == ORC_SYM_UPPER"),
    "grad_csc_transposed": ("g[k] = -(lambda[c] * x[r]);", "g[k] = -(lambda[r] * x[c]);"),
    "grad_sign": ("        g[k] = -(lambda[r] * x[c]);\n      }\n    }", "        g[k] = lambda[r] * x[c];\n      }\n    }"),
    "element_grad_drops_weight": ("if (p >= 0) s += w[e * m + k] * g[p];", "if (p >= 0) s += g[p];"),
    "assemble_drops_coefficient": ("s += tw[k] * coef[telem[k]];", "s += tw[k];"),
    "ru_drops_update": ("        x[i] += (double)d[i];\n        d[i] = 0.0f;", "        d[i] = 0.0f;"),
    "ru_keeps_correction": ("        x[i] += (double)d[i];\n        d[i] = 0.0f;", "        x[i] += (double)d[i];"),
    "ru_replacement_sign": ("r64[i] = b[i] - r64[i];\n      rel = sqrt(orc_dot(n, r64, r64)) / nb;\n      ++updates;",
                            "r64[i] = r64[i] - b[i];\n      rel = sqrt(orc_dot(n, r64, r64)) / nb;\n      ++updates;"),
    "ru_alpha_inverted": ("const float alpha = rr / pq;", "const float alpha = pq / rr;"),
    "ru_restarts_direction": ("      rmax = sqrtf(rr_new);\n    }",
                              "      rmax = sqrtf(rr_new);\n      for (int64_t i = 0; i < n; ++i) p[i] = 0.0f;\n    }"),
    "ru_threshold_never_reset": ("      rmax = sqrtf(rr_new);\n    }", "    }"),
    "pipelined_z_drops_beta": ("z[i] = (first ? 0.0 : beta * z[i]) + q[i];", "z[i] = q[i];"),
    "pipelined_plain_denominator": ("const double den = first ? delta : delta - beta * gamma / alpha_old;",
                                    "const double den = delta;"),
    "pipelined_w_sign": ("w[i] -= alpha * z[i];", "w[i] += alpha * z[i];"),
    "pipelined_s_uses_r": ("s[i] = (first ? 0.0 : beta * s[i]) + w[i];", "s[i] = (first ? 0.0 : beta * s[i]) + r[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "mut.so")
        open(c, "w").write(mutated)
        oracle.compile_oracle(c, so)
        lib = oracle.load(so)
        failures = []
        for check in ALL_CHECKS:
            try:
                check(lib)
            except (AssertionError, FloatingPointError, ValueError, OverflowError) as e:  # noqa: PERF203
                failures.append((check.__name__, str(e)[:80]))
        assert failures, f"mutant {name} survived every pin"
