"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of ``oracle/bltc_oracle.c`` (never in the
committed file), builds it with the same flags, and runs the fast oracle pins against it in
a subprocess.  The pins must fail for every mutant, and pass for the unmodified copy.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "bltc_oracle.c")

# (name, text in the source, replacement[, occurrence, occurrences]): one mistake each.  An
# anchor that occurs more than once names which occurrence is replaced and how many there are.
MUTANTS = [
    ("dropped_dz_term", "double r2 = dx * dx + dy * dy + dz * dz;", "double r2 = dx * dx + dy * dy;"),
    ("yukawa_sign", "exp(-kappa * r) / r", "exp(kappa * r) / r"),
    ("split_on_midpoint_low", "!(b->c[d][t->perm[i]] < mid[d])", "!(b->c[d][t->perm[i]] <= mid[d])"),
    ("aspect_factor_two", "L[d] * 1.4142135623730951 >= Lmax", "L[d] * 2.0 >= Lmax"),
    ("unstable_partition", "for (int64_t i = begin; i < begin + count; ++i)\n            if (b->oct[i] == o)",
     "for (int64_t i = begin + count - 1; i >= begin; --i)\n            if (b->oct[i] == o)"),
    ("radius_full_extent", "h[d] = 0.5 * (hi[d] - lo[d]);", "h[d] = (hi[d] - lo[d]);"),
    ("cheb_endpoints_swapped", "s[0] = hi;\n    s[degree] = lo;", "s[0] = lo;\n    s[degree] = hi;"),
    ("weight_sign", "w[k] = ((k % 2) ? -1.0 : 1.0) * delta;", "w[k] = delta;"),
    ("no_exact_hit", "if (fabs(y - s[k]) < DBL_MIN) {", "if (0) {"),
    ("qhat_transposed", "qh[(k1 * n1 + k2) * n1 + k3] += a1[k1]", "qh[(k3 * n1 + k2) * n1 + k1] += a1[k1]"),
    ("far_field_uses_wrong_axis", "s1[k1], s2[k2], s3[k3], &g))", "s1[k1], s2[k3], s3[k2], &g))"),
    ("self_pair_not_skipped", "if (r2 == 0.0) return 0;", "if (r2 < 0.0) return 0;"),
    ("mac_ignores_size", "int size_ok = c->P < c->st->count[C];", "int size_ok = 1;"),
    # cluster-particle variant
    ("cp_point_potential_axes", "s1[k1], s2[k2], s3[k3], sx[j], sy[j],", "s1[k1], s2[k3], s3[k2], sx[j], sy[j],"),
    # cluster-cluster variant
    ("cc_source_grid_axes", "t1[k1], t2[k2], t3[k3], s1[m1],\n                                                  s2[m2], s3[m3], &g))",
     "t1[k1], t2[k2], t3[k3], s1[m1],\n                                                  s3[m3], s2[m2], &g))"),
    ("cc_cp_target_grid_axes", "t1[k1], t2[k2], t3[k3], sx[j], sy[j],\n                                          sz[j], &g))",
     "t1[k1], t3[k3], t2[k2], sx[j], sy[j],\n                                          sz[j], &g))"),
    # barycentric Hermite treecode
    ("hermite_H_sign", "h[j] = (1.0 - 2.0 * dl * (y - s[j])) * l2;", "h[j] = (1.0 + 2.0 * dl * (y - s[j])) * l2;"),
    ("hermite_K_dropped", "k[j] = (y - s[j]) * l2;", "k[j] = 0.0 * l2;"),
    ("hermite_G2_yukawa_term", "g[2] = e * (3.0 + 3.0 * kr + kr * kr)", "g[2] = e * (3.0 + 2.0 * kr + kr * kr)"),
    ("hermite_derivative_axis", "if (a & 4) p = p * d[0];", "if (a & 4) p = p * d[2];"),
    ("hermite_charge_axis", "const double* f1 = (a & 4) ? kk[0] : h[0];", "const double* f1 = (a & 1) ? kk[0] : h[0];"),
    # absolute-value sums (the scale of the per-target parity bars)
    ("direct_sum_abs_of_g_only",
     "            acc_abs = acc_abs + fabs(g * sq[j]);\n        }\n        phi[i] = acc;",
     "            acc_abs = acc_abs + fabs(g) * sq[j];\n        }\n        phi[i] = acc;"),
    ("direct_sum_abs_doubled",
     "            acc_abs = acc_abs + fabs(g * sq[j]);\n        }\n        phi[i] = acc;",
     "            acc_abs = acc_abs + 2.0 * fabs(g * sq[j]);\n        }\n        phi[i] = acc;"),
    ("far_field_abs_dropped",
     "                    acc_abs = acc_abs + fabs(term);\n                }\n        c->phi[t] = acc;",
     "                    acc_abs = acc_abs + 0.0 * fabs(term);\n                }\n        c->phi[t] = acc;"),
    ("near_field_abs_signed",
     "            double term = g * c->sq[j];\n            acc = acc + term;\n            acc_abs = acc_abs + fabs(term);",
     "            double term = g * c->sq[j];\n            acc = acc + term;\n            acc_abs = acc_abs + term;"),
    ("cp_near_abs_signed",
     "                acc_abs = acc_abs + fabs(g * sq[j]);\n            }\n        }\n        int64_t chain[128];",
     "                acc_abs = acc_abs + g * sq[j];\n            }\n        }\n        int64_t chain[128];"),
    ("cp_point_abs_signed", "phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc_abs;",
     "phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc;", 0, 2),
    ("cp_interpolant_abs_signed", "acc_abs = acc_abs + fabs(l) * phat_abs[T * P + k];",
     "acc_abs = acc_abs + l * phat_abs[T * P + k];", 0, 2),
    ("cc_point_abs_signed", "phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc_abs;",
     "phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc;", 1, 2),
    ("cc_interpolant_abs_dropped", "acc_abs = acc_abs + fabs(l) * phat_abs[T * P + k];",
     "acc_abs = acc_abs + 0.0 * phat_abs[T * P + k];", 1, 2),
    ("cc_pc_abs_dropped",
     "                            acc_abs = acc_abs + fabs(term);\n                        }\n            }\n            for (int64_t e = off[3][T]",
     "                            acc_abs = acc_abs + 0.0 * fabs(term);\n                        }\n            }\n            for (int64_t e = off[3][T]"),
    ("hermite_far_abs_dropped",
     "                            acc_abs = acc_abs + fabs(term);\n                        }\n                    }\n            c->phi[t] = acc;",
     "                            acc_abs = acc_abs + 0.0 * fabs(term);\n                        }\n                    }\n            c->phi[t] = acc;"),
    ("hermite_near_abs_signed",
     "                const double term = dg[0] * c->q[j];\n                acc = acc + term;\n                acc_abs = acc_abs + fabs(term);",
     "                const double term = dg[0] * c->q[j];\n                acc = acc + term;\n                acc_abs = acc_abs + term;"),
]

FAST = "not decays and not band and not degenerates"


def _run_pins(tmp_path, text):
    src = tmp_path / "m.c"
    src.write_text(text)
    lib = tmp_path / "libm.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-I", os.path.join(ROOT, "oracle"), "-o", str(lib), str(src), "-lm"],
                   check=True, capture_output=True)
    env = dict(os.environ, BLTC_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-k", FAST],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode


def test_unmodified_copy_passes(tmp_path):
    with open(SRC) as f:
        assert _run_pins(tmp_path, f.read()) == 0


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, mutant):
    name, old, new = mutant[:3]
    which, count = mutant[3:] if len(mutant) > 3 else (0, 1)
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == count, f"mutation anchor for {name} not found {count} time(s)"
    at = -1
    for _ in range(which + 1):
        at = text.index(old, at + 1)
    mutated = text[:at] + new + text[at + len(old):]
    assert _run_pins(tmp_path, mutated) != 0, f"pins missed mutant {name}"
