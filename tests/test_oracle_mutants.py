"""Strength of the oracle pins: plant one plausible mistake at a time in a copy
of oracle/cqk_oracle.c (on the CPU), and check that the pin suites fail for
every mutant.  The unmodified oracle passes the same suites (the other test
files)."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cqk_oracle.c")
PINS = ["tests/test_oracle_general.py", "tests/test_oracle_simplex.py", "tests/test_oracle_grad.py",
        "tests/test_oracle_warm.py"]

# (name, original text, mutated text): each must occur exactly once
MUTANTS = [
    ("xopt_sign", "double t = (b * lam + a) / d;", "double t = (b * lam - a) / d;"),
    ("phi_drops_b", "phi += (long double)b[i] * (long double)xi;", "phi += (long double)xi;"),
    ("slope_plus_tie", "if (lo <= lam && lam < up) dp += w;", "if (lo < lam && lam < up) dp += w;"),
    ("slope_weight", "double w = b[i] * b[i] / d[i];", "double w = b[i] / d[i];"),
    ("lambda0_term", "s += (long double)(b[i] * a[i] / d[i]);\n        q += (long double)(b[i] * b[i] / d[i]);\n    }\n    return",
     "s += (long double)(a[i] / d[i]);\n        q += (long double)(b[i] * b[i] / d[i]);\n    }\n    return"),
    ("breakpoint_sign", "return (d * l - a) / b; }", "return (d * l + a) / b; }"),
    ("secant_denominator", "else { next = lower - (phi_lower - r) * (upper - lower) / (phi_upper - phi_lower); (*nsecant)++; }\n            } else {\n                int found;\n                (*bpsearch)++;\n                next = cqko_breakpoint(n, a, b, d, l, u, lower, +1, &found);",
     "else { next = lower - (phi_lower - r) * (upper - lower) / (phi_upper + phi_lower); (*nsecant)++; }\n            } else {\n                int found;\n                (*bpsearch)++;\n                next = cqko_breakpoint(n, a, b, d, l, u, lower, +1, &found);"),
    ("segment_fixed_bound", "if (m <= lo) fixed += (long double)b[i] * l[i];", "if (m <= lo) fixed += (long double)b[i] * u[i];"),
    ("alg2_count", "lam = (r - S - yj) / (double)(nJ + 1);\n            if (lam < r - yj) {", "lam = (r - S - yj) / (double)(nJ + 2);\n            if (lam < r - yj) {"),
    ("alg2_restart", "lam = r - yj;\n            }\n        }\n        if (trace)", "lam = r + yj;\n            }\n        }\n        if (trace)"),
    ("alg4_slope", "else { upper = lam; step = -g / f[2]; }", "else { upper = lam; step = -g / f[1]; }"),
    ("alg4_stop", "if (g <= 0.0) { *stop = STOPR_BELOW; return ORC_OK; }", "if (g < -1.0) { *stop = STOPR_BELOW; return ORC_OK; }"),
    ("sort_simplex_rho", "if ((long double)s[j] - (cum - r) / (long double)(j + 1) > 0.0L)", "if ((long double)s[j] - (cum + r) / (long double)(j + 1) > 0.0L)"),
    ("alg3_update", "lam = (r - S) / (double)size_after;", "lam = (r + S) / (double)size_after;"),
    ("warm_free_test", "if (l[i] < xbar[i] && xbar[i] < u[i]) {", "if (l[i] <= xbar[i] && xbar[i] < u[i]) {"),
    ("warm_support_test", "if (i >= 0 && (l1 ? xbar[i] != 0.0 : xbar[i] > 0.0)) idx[p++] = i;",
     "if (i >= 0 && (l1 ? xbar[i] != 0.0 : xbar[i] >= 0.0)) idx[p++] = i;"),
    ("warm_fallback", "return fmax(r / (double)n, -y1);", "return fmax(r / (double)n, y1);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "mut.c")
        so = os.path.join(td, "libmut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", so, c, "-lm"])
        env = dict(os.environ, CQK_ORACLE_SO=so)
        res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                             cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert res.returncode != 0, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"
