"""The oracle pins must fail on a plausibly wrong oracle.

Each case plants one mistake in a scratch copy of oracle/sun_oracle.c (CPU
only), builds it, and runs the pin suites against it in a subprocess: at least
one pin has to fail.  A substitution that no longer applies to the source fails
this test too, so the list follows the oracle's text.
"""
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    # heatbath strength without the factor 2 of alpha = 2 beta k / Nc
    "alpha_half": (r"double alpha = 2\.0 \* beta \* k / nc;", "double alpha = beta * k / nc;"),
    # staple forward term without the dagger on U_nu(x+mu)
    "staple_no_dagger": (r"mat_dag\(nc, link_c\(U, nc, V, nu, xpmu\), D\);\n    mat_mul\(nc, T1, D, T2\);",
                         "mat_mul(nc, T1, link_c(U, nc, V, nu, xpmu), T2);"),
    # staple backward term at x+nu instead of x-nu
    "staple_wrong_site": (r"int64_t xmnu = hop\(dims, lex, nu, -1\);", "int64_t xmnu = hop(dims, lex, nu, +1);"),
    # overrelaxation with vhat^2 instead of (vhat^+)^2
    "or_no_dagger": (r"mat_mul\(2, Vhd, Vhd, A\);", "mat_mul(2, Vh, Vh, A);"),
    # Kennedy-Pendleton rate alpha instead of 2 alpha
    "kp_rate": (r"/ \(2\.0 \* alpha\);", "/ alpha;"),
    # Creutz inversion with the wrong scale
    "creutz_scale": (r"1\.0 \+ log1p\(-r\[0\] \* e\) / alpha :",
                     "1.0 + log1p(-r[0] * e) / (2.0 * alpha) :"),
    # plaquette with U_nu(x+mu)^+ in place of U_mu(x+nu)^+
    "plaquette_swapped_link": (r"mat_dag\(nc, link_c\(U, nc, V, mu, hop\(dims, lex, nu, \+1\)\), D\);",
                               "mat_dag(nc, link_c(U, nc, V, nu, hop(dims, lex, mu, +1)), D);"),
    # subgroup update applied to columns instead of rows
    "cm_columns": (r"U\[i \* nc \+ c\] = A\[0\] \* ui \+ A\[1\] \* uj;\n        U\[j \* nc \+ c\] = A\[2\] \* ui \+ A\[3\] \* uj;",
                   "U[i * nc + c] = A[0] * ui + A[2] * uj;\n        U[j * nc + c] = A[1] * ui + A[3] * uj;"),
    # reunitarization without the determinant phase
    "reunit_no_phase": (r"for \(int c = 0; c < nc; \+\+c\) U\[\(nc - 1\) \* nc \+ c\] \*= phase;", ""),
    # Polyakov loop over the x direction instead of t
    "polyakov_wrong_dir": (r"mat_copy\(nc, link_c\(U, nc, V, 3, xs\), P\);", "mat_copy(nc, link_c(U, nc, V, 0, xs), P);"),
    # one wrong Philox multiplier
    "philox_constant": (r"M1 = 0xCD9E8D57u", "M1 = 0xCD9E8D59u"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(name, tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    pattern, repl = MUTANTS[name]
    src = open(os.path.join(ROOT, "oracle", "sun_oracle.c")).read()
    mutated, n = re.subn(pattern, lambda m: repl, src, count=1)
    assert n == 1, f"mutation {name} no longer matches the oracle source"
    shutil.copy(os.path.join(ROOT, "oracle", "sun_oracle.h"), tmp_path / "sun_oracle.h")
    (tmp_path / "m.c").write_text(mutated)
    lib = tmp_path / "m.so"
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(lib), str(tmp_path / "m.c"), "-lm"], check=True, capture_output=True)
    env = dict(os.environ, SUN_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        os.path.join(ROOT, "tests", "test_oracle_updates.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode != 0, f"no pin caught mutation {name}:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout
