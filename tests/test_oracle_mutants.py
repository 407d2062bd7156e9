"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case compiles a copy of oracle/fp_oracle.c with one deliberate slip in the rate path (Eqs. tao0 and
4phgamma, the Gaussian of Sec. 2.4 and the broadening of App. B), loads it in a child pytest run through
FP_ORACLE_LIB, and requires the pin tests to fail.  A control run with the unmodified source must pass,
so a failure is the slip's doing.  Everything runs on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fp_oracle.c")
PINS = ["tests/test_oracle_delta.py", "tests/test_oracle_rates.py::test_single_q_closed_form_in_si_units"]

# (name, text in oracle_rates4, replacement): the first occurrence of the text is in oracle_rates4
MUTANTS = [
    ("gaussian-without-sqrt-pi", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / (sigma * sigma)) / sigma"),
    ("gaussian-sigma-not-squared", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / sigma) / (sqrt(M_PI) * sigma)"),
    ("gaussian-normalised-by-sigma-squared", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma * sigma)"),
    ("dq-without-1/N", "return cbrt(fabs(det) / (double)p->nq);", "return cbrt(fabs(det));"),
    ("per-axis-without-1/N_a", "pa[a] = ((dx * b[0] + dy * b[1]) + dz * b[2]) / (double)p->grid[a];",
     "pa[a] = ((dx * b[0] + dy * b[1]) + dz * b[2]);"),
    ("per-axis-without-1/3", "double s = ((pa[0] * pa[0] + pa[1] * pa[1]) + pa[2] * pa[2]) / 3.0;",
     "double s = ((pa[0] * pa[0] + pa[1] * pa[1]) + pa[2] * pa[2]);"),
    ("prefactor-1/N-not-1/N^2", "(8.0 * (double)nq * (double)nq)", "(8.0 * (double)nq)"),
    ("window-without-sigma-min", "const double sw = (sigma < sigma_min) ? sigma_min : sigma;",
     "const double sw = sigma;"),
    ("sigma-from-the-wrong-leg", "orc_sigma(&P, vel + 3 * (q2 * nb + j2), vel + 3 * (q3 * nb + j3)",
     "orc_sigma(&P, vel + 3 * (q1 * nb + j1), vel + 3 * (q3 * nb + j3)"),
]


def _build(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-D_GNU_SOURCE", "-o", so, c, "-lm"])
    return so


def _run_pins(so):
    env = dict(os.environ, FP_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_control_build_passes_the_pins(tmp_path):
    with open(SRC) as f:
        text = f.read()
    rc, out = _run_pins(_build(text, str(tmp_path), "control"))
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(tmp_path, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert old in text, "the oracle no longer contains the text this case mutates"
    mutated = text.replace(old, new, 1)
    rc, out = _run_pins(_build(mutated, str(tmp_path), "mutant"))
    assert rc == 1, f"{name}: the pins did not fail (pytest rc {rc})\n{out}"
