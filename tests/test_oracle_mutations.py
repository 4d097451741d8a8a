"""The pins of the oracle catch plausible mistakes: each case plants one
mistake in a copy of oracle/helk_oracle.c (a dropped term, a flipped sign, a
wrong index or constant, a transposed operand), builds it, and runs the
oracle's pin tests against it in a subprocess; at least one pin must fail.
Nothing here touches a GPU."""
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "helk_oracle.c")
PINS = ["tests/test_oracle_voigt.py", "tests/test_oracle_lines.py", "tests/test_oracle_kdist.py"]

# (name, original text, planted mistake)
MUTATIONS = [
    ("916 drops the sinc term", "K += (2.0 * h * x / OR_PI) * ex2 * sin(xy) * sinc;", ""),
    ("916 flips the S1 sign", "-y * c2xy * ex2 * s1", "+y * c2xy * ex2 * s1"),
    ("916 wrong S3 index", "exp(-((nh - x) * (nh - x)))", "exp(-((nh - x) * (nh + x)))"),
    ("916 wrong step", "#define OR_A916_H     0.5", "#define OR_A916_H     0.6"),
    ("GH3 wrong outer weight", "w1 = OR_SQRTPI / 6.0", "w1 = OR_SQRTPI / 3.0"),
    ("GH3 node sign", "d2 = (x + t) * (x + t) + y2", "d2 = (x - t) * (x - t) + y2"),
    ("GH1 drops y^2", "(OR_SQRTPI / (x * x + y * y))", "(OR_SQRTPI / (x * x))"),
    ("GH3 threshold", "#define OR_R2_GH3    100.0", "#define OR_R2_GH3    30.0"),
    ("Doppler drops ln2", "sqrt(2.0 * OR_LN2 * OR_KB * T", "sqrt(2.0 * OR_KB * T"),
    ("Doppler mass units", "/ (mass * OR_AMU)) / OR_CLIGHT", "/ (mass)) / OR_CLIGHT"),
    ("Lorentz self pressure", "pself = 0.5 * P;", "pself = P;"),
    ("Lorentz T exponent", "sqrt(OR_T0 / T)", "sqrt(T / OR_T0)"),
    ("Boltzmann sign", "exp(-OR_C2 * E / T + OR_C2 * E / OR_T0)",
     "exp(OR_C2 * E / T - OR_C2 * E / OR_T0)"),
    ("strength ignores Q ratio", "S = S * q_ratio * boltz * stim;", "S = S * boltz * stim;"),
    ("pressure shift ignores P", "r->nu0p = nu0 + delta * P;", "r->nu0p = nu0 + delta;"),
    ("window lower bound", "lo = ceil((r->nu0p - r->cut - nu_min) / dnu);",
     "lo = floor((r->nu0p - r->cut - nu_min) / dnu);"),
    ("Lorentz cutoff cap", "fmin(cut_value * r->gL, cut_cap)", "fmax(cut_value * r->gL, cut_cap)"),
    ("u divides by ku", "double u    = (nu_i - r->nu0p) * r->ku;", "double u    = (nu_i - r->nu0p) / r->ku;"),
    ("accumulation overwrites", "acc[i - c->g0] += r->Sp * H;", "acc[i - c->g0] = r->Sp * H;"),
    ("per-line weight ignored", "if (L->weight) S = S * L->weight[l];", ""),
    ("per-line mass ignored", "if (L->mass) mass = L->mass[l];", ""),
    ("k-abscissa not midpoint", "double g = ((double)j + 0.5) / (double)nb;", "double g = ((double)j) / (double)nb;"),
    ("Chebyshev recurrence sign", "row[c] = 2.0 * t * row[c - 1] - row[c - 2];",
     "row[c] = 2.0 * t * row[c - 1] + row[c - 2];"),
    ("QR back substitution transposed", "s2 -= A[c * ncheb + cc] * coef[cc];", "s2 -= A[cc * ncheb + c] * coef[cc];"),
    ("sort descending", "return (a > b) - (a < b);", "return (a < b) - (a > b);"),
    ("transmission divides by m", "s += exp(-k[j] * m[i]);", "s += exp(-k[j] / m[i]);"),
    ("kappa floor ignored", "double kv = k[j] > kappa_floor ? k[j] : kappa_floor;", "double kv = k[j];"),
]


def _run_mutant(case):
    name, old, new = case
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %s" % name
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "m.so")
        open(c, "w").write(src.replace(old, new, 1))
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-std=c99", "-D_GNU_SOURCE", "-fPIC", "-shared",
                        "-o", so, c, "-lm", "-lpthread"], check=True)
        env = dict(os.environ, HELK_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return name, r.returncode


def test_pins_catch_planted_mistakes():
    control = ("unchanged source", "#define OR_T0", "#define OR_T0")
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(_run_mutant, [control] + MUTATIONS))
    assert results[0][1] == 0, "the harness fails an unchanged oracle"
    survived = [name for name, rc in results[1:] if rc == 0]
    assert not survived, "mistakes no pin caught: %s" % survived
