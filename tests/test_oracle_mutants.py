"""Mutation tests for the oracle's pins: plant a plausible mistake in a copy of
the C oracle (on the CPU), rebuild it, and require that at least one pin
catches it.  Each mutant runs in a child process so a crash counts as caught."""
import os
import subprocess
import sys
import tempfile

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ttv_oracle.c")

MUTANTS = {
    "dropped_term": ("            sum = 0.0;\n            comp = 0.0;\n        }",
                     "            sum = 0.0;\n            comp = 0.0;\n            continue;\n        }"),
    "wrong_sign": ("if (in_s[m]) p = p * vec_of_mode[m][subs[k * d + m]];",
                   "if (in_s[m]) p = -p * vec_of_mode[m][subs[k * d + m]];"),
    "wrong_vector_index": ("if (in_s[m]) p = p * vec_of_mode[m][subs[k * d + m]];",
                           "if (in_s[m]) p = p * vec_of_mode[m][subs[k * d + 0] % shape[m]];"),
    "product_skips_last_mode": ("for (int32_t m = 0; m < d; ++m)\n            if (in_s[m]) p",
                                "for (int32_t m = 0; m < d - 1; ++m)\n            if (in_s[m]) p"),
    "transposed_output_subs": ("gsubs[g * ctx.nr + j] = subs[k * d + ctx.r[j]];",
                               "gsubs[g * ctx.nr + j] = subs[k * d + ctx.r[ctx.nr - 1 - j]];"),
    "descending_order": ("if (a < b) return -1;\n        if (a > b) return 1;",
                         "if (a < b) return 1;\n        if (a > b) return -1;"),
    "group_on_first_mode_only": ("for (int32_t j = 0; j < c->nr; ++j)\n        if (c->subs",
                                 "for (int32_t j = 0; j < c->nr && j < 1; ++j)\n        if (c->subs"),
    "no_compensation": ("double s = sum + t[k];\n        if (fabs(sum) >= fabs(t[k])) comp += (sum - s) + t[k];\n        else                         comp += (t[k] - s) + sum;",
                        "double s = sum + t[k];"),
    "first_mode_never_survives": ("for (int32_t m = 0; m < d; ++m)\n        if (!in_s[m]) ctx.r[ctx.nr++] = m;",
                                  "for (int32_t m = 1; m < d; ++m)\n        if (!in_s[m]) ctx.r[ctx.nr++] = m;"),
    "dense_column_major": ("lin = lin * out->shape[j] + gsubs[q * ctx.nr + j];",
                           "lin = lin + gsubs[q * ctx.nr + j] * (j == 0 ? 1 : out->shape[j - 1]);"),
}

MTTKRP_MUTANTS = {
    "mttkrp_skips_a_mode": ("if (m != mode) t = t * factors[m][subs[k * d + m] * rank + r];",
                            "if (m != mode && m != d - 1) t = t * factors[m][subs[k * d + m] * rank + r];"),
    "mttkrp_wrong_factor_row": ("if (m != mode) t = t * factors[m][subs[k * d + m] * rank + r];",
                                "if (m != mode) t = t * factors[m][(subs[k * d + m] % shape[m]) * rank + 0];"),
    "mttkrp_wrong_output_row": ("const int64_t i = subs[k * d + mode];",
                                "const int64_t i = subs[k * d + mode] == 0 ? 0 : subs[k * d + mode] - 1;"),
    "mttkrp_factor_read_column_major": ("if (m != mode) t = t * factors[m][subs[k * d + m] * rank + r];",
                                        "if (m != mode) t = t * factors[m][r * shape[m] + subs[k * d + m]];"),
    "mttkrp_no_compensation": ("if (fabs(*sum) >= fabs(t)) *c += (*sum - s) + t;\n            else                       *c += (t - s) + *sum;",
                               ""),
}

DENSE_MUTANTS = {
    "dense_shifted_index": ("const double t = a[i * sa] * b[i];",
                            "const double t = a[i * sa] * b[i + 1 < n ? i + 1 : i];"),
    "dense_no_compensation": ("if (fabs(sum) >= fabs(t)) comp += (sum - s) + t;\n        else                      comp += (t - s) + sum;",
                              ""),
    "matvec_transposed": ("y[i] = neumaier_sum_products(A + i * stride_row, stride_col, x, n2);",
                          "y[i] = neumaier_sum_products(A + (i % n2) * stride_col, stride_row, x, n2 < n1 ? n2 : n1);"),
    "matvec_skips_last_column": ("y[i] = neumaier_sum_products(A + i * stride_row, stride_col, x, n2);",
                                 "y[i] = neumaier_sum_products(A + i * stride_row, stride_col, x, n2 > 1 ? n2 - 1 : n2);"),
}

RUNNER_DENSE = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins as P
lib = oracle.load_library({lib!r})
dot = lambda *a, **k: oracle.dot(*a, lib=lib, **k)
mv = lambda *a, **k: oracle.matvec(*a, lib=lib, **k)
g = lambda *a, **k: oracle.ttv(*a, lib=lib, **k)
failed = []
for c in P.DENSE_CHECKS:
    try:
        c(dot, mv, g)
    except Exception as e:
        failed.append(c.__name__)
print("FAILED", len(failed), failed)
"""

RUNNER_MTTKRP = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins as P
lib = oracle.load_library({lib!r})
f = lambda *a, **k: oracle.mttkrp(*a, lib=lib, **k)
g = lambda *a, **k: oracle.ttv(*a, lib=lib, **k)
failed = []
for c in P.MTTKRP_CHECKS:
    try:
        c(f, g)
    except Exception as e:
        failed.append(c.__name__)
print("FAILED", len(failed), failed)
"""

RUNNER = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle, oracle_pins as P
lib = oracle.load_library({lib!r})
f = lambda *a, **k: oracle.ttv(*a, lib=lib, **k)
failed = []
for c in P.ALL_CHECKS:
    try:
        c(f)
    except Exception as e:
        failed.append(c.__name__)
print("FAILED", len(failed), failed)
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    with tempfile.TemporaryDirectory() as td:
        msrc = os.path.join(td, "mutant.c")
        open(msrc, "w").write(src.replace(old, new))
        lib = oracle.compile_library(msrc, os.path.join(td, "libmutant.so"))
        code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    caught = r.returncode != 0 or ("FAILED" in r.stdout and "FAILED 0 " not in r.stdout)
    assert caught, f"mutant {name} survived every pin: {r.stdout} {r.stderr[-500:]}"


@pytest.mark.parametrize("name", sorted(MTTKRP_MUTANTS))
def test_mttkrp_pins_catch_mutant(name):
    old, new = MTTKRP_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    with tempfile.TemporaryDirectory() as td:
        msrc = os.path.join(td, "mutant.c")
        open(msrc, "w").write(src.replace(old, new))
        lib = oracle.compile_library(msrc, os.path.join(td, "libmutant.so"))
        code = RUNNER_MTTKRP.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    caught = r.returncode != 0 or ("FAILED" in r.stdout and "FAILED 0 " not in r.stdout)
    assert caught, f"mutant {name} survived every pin: {r.stdout} {r.stderr[-500:]}"


@pytest.mark.parametrize("name", sorted(DENSE_MUTANTS))
def test_dense_pins_catch_mutant(name):
    old, new = DENSE_MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    with tempfile.TemporaryDirectory() as td:
        msrc = os.path.join(td, "mutant.c")
        open(msrc, "w").write(src.replace(old, new))
        lib = oracle.compile_library(msrc, os.path.join(td, "libmutant.so"))
        code = RUNNER_DENSE.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    caught = r.returncode != 0 or ("FAILED" in r.stdout and "FAILED 0 " not in r.stdout)
    assert caught, f"mutant {name} survived every pin: {r.stdout} {r.stderr[-500:]}"
