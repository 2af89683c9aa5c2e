"""Plant plausible mistakes in copies of the oracle (on the CPU) and check
that the pins of test_oracle_pins.py catch every one of them."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    "dropped_y_normalisation": ("- d * (LN_SQRT_2PI + log(h1))\n                               - (LN_SQRT_2PI + log(h2));",
                                "- d * (LN_SQRT_2PI + log(h1));"),
    "wrong_sign_in_y_exponent": ("e[i] = -dx2[i] / (2.0 * h1 * h1) - dy2[i] / (2.0 * h2 * h2);",
                                 "e[i] = -dx2[i] / (2.0 * h1 * h1) + dy2[i] / (2.0 * h2 * h2);"),
    "swapped_bandwidth_roles": ("e[i] = -dx2[i] / (2.0 * h1 * h1) - dy2[i] / (2.0 * h2 * h2);",
                                "e[i] = -dx2[i] / (2.0 * h2 * h2) - dy2[i] / (2.0 * h1 * h1);"),
    "leave_one_out_dropped": ("if (i != j) s += exp(e[i] - m);", "s += exp(e[i] - m);"),
    "x_constant_only_in_B": ("const double lnB = lse_excl(e, J->N, j) - d * (LN_SQRT_2PI + log(h1));",
                             "const double lnB = lse_excl(e, J->N, j);"),
    "gradient_h2_sign": ("out[2] = (sAy / sA) / (J->h2 * J->h2) - 1.0;",
                         "out[2] = (sAy / sA) / (J->h2 * J->h2) + 1.0;"),
    "density_missing_constant": ("double lnf = mA + log(sA) - lnB - (LN_SQRT_2PI + log(J->h2));",
                                 "double lnf = mA + log(sA) - lnB;"),
    "sd_without_ddof": ("double sd = sqrt(nm_val(&v) / (double)(N - 1));",
                        "double sd = sqrt(nm_val(&v) / (double)N);"),
    "eq3_wrong_count": ("L_eq3[c] = nm_val(&b) / (double)N - log((double)(N - 1));",
                        "L_eq3[c] = nm_val(&b) / (double)N - log((double)N);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: " + name
    mutant = tmp_path / "oracle.c"
    mutant.write_text(src.replace(old, new))
    env = dict(os.environ, ORACLE_SRC=str(mutant))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, "the pins did not catch mutation %s" % name
    assert "failed" in r.stdout
