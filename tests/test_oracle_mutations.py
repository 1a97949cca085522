"""The oracle's pins catch plausible mistakes: each mutation below is planted
in a temporary copy of the oracle source (never in the committed oracle),
compiled, and the pins are run against it until one fails."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pthr_oracle.c")

MUTANTS = [
    ("dropped neighbour term in the local field", "for (int k = 0; k < 6; k++) h += J[bond[k]]",
     "for (int k = 0; k < 5; k++) h += J[bond[k]]"),
    ("backward x bond attached to the wrong site", "bond[1] = 0 * V + nb[1];", "bond[1] = 0 * V + i;"),
    ("Metropolis exponent sign", "p = exp(-beta * dEi);", "p = exp(beta * dEi);"),
    ("heat-bath exponent sign", "p = 1.0 / (1.0 + exp(-2.0 * beta * h));",
     "p = 1.0 / (1.0 + exp(2.0 * beta * h));"),
    ("PT energy difference transposed", "double delta = (beta[k] - beta[k + 1]) * (E[k] - E[k + 1]);",
     "double delta = (beta[k] - beta[k + 1]) * (E[k + 1] - E[k]);"),
    ("ACU sign drawn per site, not per cluster",
     "uint32_t w = rng_word(seed, (uint32_t)lab[i], pair_id, emcs, TAG_ACU, 0);",
     "uint32_t w = rng_word(seed, (uint32_t)i, pair_id, emcs, TAG_ACU, 0);"),
    ("cluster rule inverted", "if (lab[w] < 0 && sa[w] * sb[w] == qv)", "if (lab[w] < 0 && sa[w] * sb[w] != qv)"),
    ("energy misses the z bonds", "        H -= J[bond[4]] * s[i] * s[nb[4]];\n", ""),
    ("link overlap uses one replica", "ql += qi * (double)(sa[nb[0]] * sb[nb[0]]);",
     "ql += qi * (double)(sa[nb[0]]);"),
    ("Philox multiplier constant", "#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F52u"),
    ("ER exchanges the youngest reservoir clone", "if (age[r] > age[best]) best = r;",
     "if (age[r] < age[best]) best = r;"),
    ("Boltzmann weight sign in the enumeration", "double w = exp(-beta * (H[st] - Hmin));",
     "double w = exp(beta * (H[st] - Hmin));"),
    ("SDY sign of the link term", "out[2] = Ha / (3.0 * V) + (1.0 - ql) / T;",
     "out[2] = Ha / (3.0 * V) + (1.0 + ql) / T;"),
    ("Box-Muller radius", "double r = sqrt(-2.0 * log(u1));", "double r = sqrt(-log(u1));"),
    ("PT skips the odd phase", "for (int ph = 0; ph < 2; ph++) {\n        for (int k = ph; k + 1 < n_temps; k += 2) {",
     "for (int ph = 0; ph < 1; ph++) {\n        for (int k = ph; k + 1 < n_temps; k += 2) {"),
    ("q^2 enumeration drops the square", "for (int b = 0; b < V; b++) q2 += C[a][b] * C[a][b];",
     "for (int b = 0; b < V; b++) q2 += C[a][b];"),
    ("e^2 accumulated as e", "o[2] += e * e;", "o[2] += e;"),
    ("q^4 accumulated as q^3", "o[7] += r[0] * r[0] * r[0] * r[0];", "o[7] += r[0] * r[0] * r[0];"),
    ("overlap accumulated as |q|", "o[3] += r[0];", "o[3] += fabs(r[0]);"),
    ("temperature grid divided by N_T", "(t_max - t_min) / (double)(n_temps - 1);",
     "(t_max - t_min) / (double)(n_temps);"),
    ("MicSA walker not debited", "        if (f) D += dE[k];\n", ""),
    ("MicSA walker credited instead of debited", "if (f) D += dE[k];", "if (f) D -= dE[k];"),
    ("MicSA energy change of a flip dropped", "if (dE_total) *dE_total += dE[k];", "if (dE_total) *dE_total += 0.0;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {name}"
    mut = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    so = tmp_path / "libmutant.so"
    c.write_text(mut)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", str(so), str(c), "-lm"])
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "oracle_mutant_runner.py")],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, f"mutation '{name}' survived every pin:\n{r.stdout}\n{r.stderr}"
