"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of ``oracle/lse_oracle.c`` (on the
CPU, in a temporary directory), builds it, and runs the pin suite against that
build; the suite has to fail.  The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lse_oracle.c")

MUTATIONS = {
    # Eq. 16's printed plus instead of Eq. 15/17's minus
    "eq16_plus": ("d += (cp - cm) * (2.0", "d += (cp + cm) * (2.0"),
    # central difference without the 1/2
    "no_half": ("return 0.5 * (row[x + 1] - row[x - 1]);",
                "return (row[x + 1] - row[x - 1]);"),
    # one-sided difference with the wrong sign at the first column
    "border_sign": ("if (x == 0) return row[1] - row[0];",
                    "if (x == 0) return row[0] - row[1];"),
    # y-gradient taken along x (transposed operand)
    "transposed": ("return 0.5 * (f[(size_t)(y + 1) * W + x] - f[(size_t)(y - 1) * W + x]);",
                   "return 0.5 * (f[(size_t)y * W + x + 1] - f[(size_t)y * W + x - 1]);"),
    # correlation instead of convolution
    "conv_flip": ("int yy = y - i;", "int yy = y + i;"),
    # tie v = 0 sent to -1
    "tie_rule": ("phi[p] = reinit ? (v_out[p] >= 0.0 ? 1.0 : -1.0) : v_out[p];",
                 "phi[p] = reinit ? (v_out[p] > 0.0 ? 1.0 : -1.0) : v_out[p];"),
    # dropped time step
    "no_dt": ("return c->phi[p] + c->dt * force_at(c, p) * sqrt(fx * fx + fy * fy);",
              "return c->phi[p] + force_at(c, p) * sqrt(fx * fx + fy * fy);"),
    # |grad phi|^2 instead of |grad phi|
    "no_sqrt": ("* sqrt(fx * fx + fy * fy);", "* (fx * fx + fy * fy);"),
    # Gaussian exponent without the factor 2
    "sigma_sq": ("/ (2.0 * sigma * sigma));", "/ (sigma * sigma));"),
    # edge indicator without the intensity scale
    "no_edge_scale": ("J[p] = edge_scale * (acc / B);", "J[p] = (acc / B);"),
    # band mean replaced by the first band
    "first_band_only": ("for (int b = 0; b < B; ++b)\n            acc += I[(size_t)b * N + p];",
                        "acc = B * I[p];"),
    # phi = 0 counted on the minus side
    "zero_side": ("if (phi[p] >= 0.0) s_plus += Ib[p];", "if (phi[p] > 0.0) s_plus += Ib[p];"),
    # normaliser taken without the absolute value
    "no_abs_norm": ("double a = fabs(region_numerator_at(c, p));",
                    "double a = region_numerator_at(c, p);"),
    # update without the LSF itself
    "no_phi_term": ("return c->phi[p] + c->dt", "return 0.0 + c->dt"),
    # replicate padding clamping to the far border
    "replicate_far_side": ("yy = yy < 0 ? 0 : H - 1;", "yy = yy < 0 ? H - 1 : 0;"),
    # Table I re-initialisation with the tie u = 0 sent to -1
    "table1_tie": ("u[p] = u[p] >= 0.0 ? 1.0 : -1.0;", "u[p] = u[p] > 0.0 ? 1.0 : -1.0;"),
    # Table I order without its re-initialisation before smoothing
    "table1_no_binarise": ("if (order == ORACLE_ORDER_TABLE1 && reinit)",
                           "if (order == ORACLE_ORDER_TABLE1 && 0)"),
    # re-initialisation one iteration early in a periodic schedule
    "reinit_phase": ("return ((n + 1) % period) == 0;", "return (n % period) == 0;"),
    # early stop when the count equals the threshold (the rule is strict)
    "stop_not_strict": ("(double)flips < early_stop_frac * (double)N",
                        "(double)flips <= early_stop_frac * (double)N"),
    # a starting value of exactly 0 counted on the minus side for sign changes
    "flip_strict_side": ("if ((v_out[p] >= 0.0) != (phi[p] >= 0.0)) ++flips;",
                         "if ((v_out[p] >= 0.0) != (phi[p] > 0.0)) ++flips;"),
    # sign changes counted against the re-initialised LSF (always 0 then)
    "flips_after_reinit": ("        st->last_flips = flips;\n",
                           "        st->last_flips = 0;\n"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    before, after = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation anchor for {name} not unique"
    mutated = tmp_path / "lse_oracle_mutant.c"
    mutated.write_text(src.replace(before, after))
    lib = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", str(lib), str(mutated), "-lm"])
    env = dict(os.environ, LSE_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p",
                        "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode != 0, f"pins did not catch mutation {name}:\n{r.stdout[-2000:]}"
