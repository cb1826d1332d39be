"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (on the CPU),
compiles it, and runs the pin tests against the mutant library: at least one
pin must fail. The real oracle is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rime_oracle.c")

# (name, text in the oracle, planted replacement)
MUTANTS = [
    ("conj on antenna p", "cplx z = (ap.E * ap.K) * conj(aq.E * aq.K);",
     "cplx z = conj(ap.E * ap.K) * (aq.E * aq.K);"),
    ("phase sign", "r.K = cos(phi) + IMAG * sin(phi);", "r.K = cos(phi) - IMAG * sin(phi);"),
    ("w term dropped", "uvw[2] * n1) / lambda", "uvw[2] * 0.0) / lambda"),
    ("n instead of n-1", "uvw[2] * n1) / lambda", "uvw[2] * (n1 + 1.0)) / lambda"),
    ("beam squared not cubed", "*E = c * c * c;", "*E = c * c;"),
    ("jinc: J0 for 2 J1(x)/x", "*E = 2.0 * j1x / x;", "*E = j0x;"),
    ("jinc: series x^2 term", "*E = 1.0 - x2 / 8.0 +", "*E = 1.0 - x2 / 4.0 +"),
    ("grad: jinc derivative J2", "*dEx = -2.0 * (2.0 * j1x / x - j0x) / (x * x);",
     "*dEx = -2.0 * (j1x / x - j0x) / (x * x);"),
    ("grad: jinc derivative series", "*dEx = -0.25 + x2 / 48.0", "*dEx = -0.5 + x2 / 48.0"),
    ("beam in wavelength", "double cnu = P->beam_c * (nu * 1e-9);",
     "double cnu = P->beam_c * lambda;"),
    ("pointing sign", "hypot(l - dl, m - dm)", "hypot(l + dl, m - dm)"),
    ("gaussian axes swapped", "double umaj = u * sin(pa) + v * cos(pa);",
     "double umaj = u * cos(pa) + v * sin(pa);"),
    ("disk exponent", "r.g = pow(1.0 + q, -1.5);", "r.g = pow(1.0 + q, -1.0);"),
    ("disk constant", "double kd = 4.0 * PI * PI;", "double kd = 2.0 * PI * PI;"),
    ("grad: disk derivative factor", "double dgdq = -1.5 * r.g / (1.0 + q);", "double dgdq = -1.5 * r.g;"),
    ("gaussian FWHM constant", "double k = PI * PI / (4.0 * log(2.0));",
     "double k = PI * PI / (2.0 * log(2.0));"),
    ("gaussian on u_p + u_q", "up[0] - uq[0], up[1] - uq[1], lambda);\n        cplx B[4];\n        brightness",
     "up[0] + uq[0], up[1] - uq[1], lambda);\n        cplx B[4];\n        brightness"),
    ("spectral ratio inverted", "double spec = pow(lambda_ref / lambda, P->alpha[s]);\n        shape_term sh = shape_factor(P, s, up[0] - uq[0], up[1] - uq[1], lambda);\n        cplx B[4];\n        brightness(stokes_of(P, t, s), B);\n        cplx z",
     "double spec = pow(lambda / lambda_ref, P->alpha[s]);\n        shape_term sh = shape_factor(P, s, up[0] - uq[0], up[1] - uq[1], lambda);\n        cplx B[4];\n        brightness(stokes_of(P, t, s), B);\n        cplx z"),
    ("stokes V sign", "B[1] = sU + IMAG * sV;", "B[1] = sU - IMAG * sV;"),
    ("stokes Q sign", "B[3] = sI - sQ;", "B[3] = sI + sQ;"),
    ("G_q not conjugated", "    mat_herm(gq, gqh);\n    mat_mul(gp, x, t);",
     "    memcpy(gqh, gq, sizeof gqh);\n    mat_mul(gp, x, t);"),
    ("gains swapped", "sandwich(gp, S, gq, V); /* eq. 1 */", "sandwich(gq, S, gp, V); /* eq. 1 */"),
    ("chi2 weight dropped", "return w * acc;", "return acc;"),
    ("chi2 imaginary part dropped", "acc += dr * dr + di * di;", "acc += dr * dr;"),
    ("time-varying brightness index", "return P->stokes + 4 * ((long)t * P->nsrc + s);",
     "return P->stokes + 4 * ((long)s * P->ntime + t);"),
    ("grad: phase derivative sign", "r.dK_dl = r.K * IMAG *", "r.dK_dl = r.K * (-IMAG) *"),
    ("grad: pa derivative sign", "r.g * (-k) * (2.0 * maj * maj * umaj * umin - 2.0 * mn * mn * umin * umaj);",
     "r.g * (-k) * (2.0 * maj * maj * umaj * umin + 2.0 * mn * mn * umin * umaj);"),
    ("grad: disk pa derivative sign", "dgdq * kd * (2.0 * maj * maj * umaj * umin - 2.0 * mn * mn * umin * umaj);",
     "dgdq * kd * (2.0 * maj * maj * umaj * umin + 2.0 * mn * mn * umin * umaj);"),
    ("grad: beam derivative factor", "*dEx = -3.0 * c * c * sinc;", "*dEx = -3.0 * c * sinc;"),
    ("grad: gain q imaginary sign", "for (int c = 0; c < 4; c++) dVi[c] = -IMAG * dVr[c];",
     "for (int c = 0; c < 4; c++) dVi[c] = IMAG * dVr[c];"),
    ("grad: alpha derivative", "* log(lambda_ref / lambda);", "* log(lambda / lambda_ref);"),
    ("reduced phase: floor for the nearest integer", "out[i] = x - nearbyint(x);", "out[i] = x - floor(x);"),
    ("reduced phase: truncation", "out[i] = x - nearbyint(x);", "out[i] = x - trunc(x);"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site not unique/found: {name}"
    mutant_c = tmp_path / "rime_oracle.c"
    mutant_c.write_text(text.replace(old, new))
    (tmp_path / "rime_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "rime_oracle.h")).read())
    so = tmp_path / "librime_mutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-o", str(so), str(mutant_c), "-lm"], check=True)
    env = dict(os.environ, RIME_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"no pin caught the planted mistake '{name}'\n{r.stdout[-2000:]}"
