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
    # Epanechnikov kernel
    "epan_support_not_truncated": ("return v > 0.0 ? v : 0.0;", "return v;"),
    "epan_constant_halved": ("return log(d + 2.0) - log(2.0) - 0.5 * d * log(M_PI) + lgamma(0.5 * d + 1.0);",
                             "return log(d + 2.0) - 0.5 * d * log(M_PI) + lgamma(0.5 * d + 1.0);"),
    "epan_ball_volume_power": ("return log(d + 2.0) - log(2.0) - 0.5 * d * log(M_PI) + lgamma(0.5 * d + 1.0);",
                               "return log(d + 2.0) - log(2.0) - d * log(M_PI) + lgamma(0.5 * d + 1.0);"),
    "epan_leave_one_out_dropped": ("if (i != j) A += epan_prof(dx2[i], h1) * epan_prof(dy2[i], h2);",
                                   "A += epan_prof(dx2[i], h1) * epan_prof(dy2[i], h2);"),
    "epan_gradient_indicator_dropped": ("const double v = dx2[i] < h1 * h1 ? 2.0 * dx2[i] / (h1 * h1) : 0.0;",
                                        "const double v = 2.0 * dx2[i] / (h1 * h1);"),
    "epan_gradient_h2_sign": ("out[2] = sA > 0.0 ? sAz / sA - 1.0 : 0.0;",
                              "out[2] = sA > 0.0 ? sAz / sA + 1.0 : 0.0;"),
    # products of fhat(.|x) (Sec. 4.2)
    "cdf_wrong_tail": ("return 0.5 * erfc(-t / sqrt(2.0));", "return 0.5 * erfc(t / sqrt(2.0));"),
    "epan_cdf_cubic_sign": ("return (2.0 + 3.0 * t - t * t * t) / 4.0;", "return (2.0 + 3.0 * t + t * t * t) / 4.0;"),
    "cond_mean_unweighted": ("S1 += wx[i] * J->y[i];", "S1 += J->y[i];"),
    "epan_density_missing_h2": ("J->f[q * J->G + g] = B > 0.0 ? A / B * exp(lc1 - log(J->h2)) : 0.0;",
                                "J->f[q * J->G + g] = B > 0.0 ? A / B * exp(lc1) : 0.0;"),
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
