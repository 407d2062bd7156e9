"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each case plants one deliberate slip in a copy of the oracle, runs the pin tests against the copy in a child
pytest process, and requires them to fail.  A control run with the unmodified copy must pass, so a failure is the
slip's doing.  Everything runs on the CPU.

* C cases compile a copy of oracle/fp_oracle.c and load it through FP_ORACLE_LIB.  They cover the rate path (Eqs.
  tao0 and 4phgamma: Bose combinations, multiplicities, the frequency product and the prefactor), the Gaussian of
  Sec. 2.4 and the broadening of App. B, the momentum rule and the vertex of Eq. V4 (phases, conjugated legs, mass
  scaling, index order), the three-phonon part (Eqs. 3phgamma and V3), the three-phonon-like phase space and the
  normal/Umklapp classification.
* Python cases copy the oracle package (with the tests and the input generators) to a scratch tree and plant the
  slip there: the harmonic modes, the RTA conductivity and the network's backward pass and Adam step.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fp_oracle.c")

DELTA = "tests/test_oracle_delta.py"
RATES = "tests/test_oracle_rates.py"
VERTEX = "tests/test_oracle_vertex.py"
RATES3 = "tests/test_oracle_rates3.py"
PHASE3 = "tests/test_oracle_phase3.py"
MODES = "tests/test_oracle_modes.py"
KAPPA = "tests/test_oracle_kappa.py"
MLP = "tests/test_oracle_mlp.py"
PINS = [DELTA, RATES + "::test_single_q_closed_form_in_si_units"]
CLOSED = [RATES + "::test_single_q_closed_form_in_si_units", RATES + "::test_detailed_balance_on_shell"]
BRUTE = [VERTEX]
UMKLAPP = [RATES + "::test_umklapp_hand_worked_cases", RATES + "::test_umklapp_reading_on_a_sheared_cell"]

# (name, text, replacement, pins): the first occurrence of the text is the one in oracle_rates4
MUTANTS = [
    ("gaussian-without-sqrt-pi", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / (sigma * sigma)) / sigma", PINS),
    ("gaussian-sigma-not-squared", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / sigma) / (sqrt(M_PI) * sigma)", PINS),
    ("gaussian-normalised-by-sigma-squared", "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma)",
     "exp(-(dw * dw) / (sigma * sigma)) / (sqrt(M_PI) * sigma * sigma)", PINS),
    ("dq-without-1/N", "return cbrt(fabs(det) / (double)p->nq);", "return cbrt(fabs(det));", PINS),
    ("per-axis-without-1/N_a", "pa[a] = ((dx * b[0] + dy * b[1]) + dz * b[2]) / (double)p->grid[a];",
     "pa[a] = ((dx * b[0] + dy * b[1]) + dz * b[2]);", PINS),
    ("per-axis-without-1/3", "double s = ((pa[0] * pa[0] + pa[1] * pa[1]) + pa[2] * pa[2]) / 3.0;",
     "double s = ((pa[0] * pa[0] + pa[1] * pa[1]) + pa[2] * pa[2]);", PINS),
    ("prefactor-1/N-not-1/N^2", "(8.0 * (double)nq * (double)nq)", "(8.0 * (double)nq)", PINS),
    ("window-without-sigma-min", "const double sw = (sigma < sigma_min) ? sigma_min : sigma;",
     "const double sw = sigma;", PINS),
    ("sigma-from-the-wrong-leg", "orc_sigma(&P, vel + 3 * (q2 * nb + j2), vel + 3 * (q3 * nb + j3)",
     "orc_sigma(&P, vel + 3 * (q1 * nb + j1), vel + 3 * (q3 * nb + j3)", PINS),
]

# (name, text, replacement, pins): each text occurs exactly once in fp_oracle.c
C_MUTANTS = [
    # Eq. 4phgamma: Bose combinations, 1/n_lambda, occupations, multiplicities of Eq. tao0, frequency product
    ("bose-recombination-form", "B = (1.0 + n1) * (1.0 + n2) * n3;", "B = (1.0 + n1) * n2 * n3;", CLOSED),
    ("bose-redistribution-form", "B = (1.0 + n1) * n2 * n3;", "B = n1 * (1.0 + n2) * n3;", CLOSED),
    ("bose-splitting-form", "B = n1 * n2 * n3;", "B = n1 * n2 * (1.0 + n3);", CLOSED),
    ("bose-without-1/n", "ORC_MULT[pr] * B / n0 * v2", "ORC_MULT[pr] * B * v2", CLOSED),
    ("occupation-without-minus-one", "return 1.0 / expm1(ORC_HBAR * w / (ORC_KB * T));",
     "return 1.0 / exp(ORC_HBAR * w / (ORC_KB * T));", CLOSED),
    ("multiplicity-splitting-1/2", "{0.5, 0.5, 1.0 / 6.0}", "{0.5, 0.5, 0.5}", CLOSED),
    ("multiplicity-recombination-1", "{0.5, 0.5, 1.0 / 6.0}", "{1.0, 0.5, 1.0 / 6.0}", CLOSED),
    ("frequency-product-without-w'''", "v2 * delta / (w * w1 * w2 * w3)", "v2 * delta / (w * w1 * w2)", CLOSED),
    ("unit-conversion-off-by-ten", "return ORC_ECHARGE / ORC_AMU * 1e20 * 1e-24;",
     "return ORC_ECHARGE / ORC_AMU * 1e20 * 1e-23;", CLOSED),
    ("prefactor-hbar-not-squared", "const double pref = M_PI * ORC_HBAR * ORC_HBAR * conv",
     "const double pref = M_PI * ORC_HBAR * conv", CLOSED),
    ("energy-difference-sign-of-q'", "double t = (s1 > 0) ? (w + w1) : (w - w1);",
     "double t = (s1 > 0) ? (w - w1) : (w + w1);", CLOSED),
    ("energy-difference-sign-of-q''", "t = (s2 > 0) ? (t + w2) : (t - w2);", "t = (s2 > 0) ? (t - w2) : (t + w2);", CLOSED),
    # momentum rule and Eq. V4
    ("momentum-sign-of-q''", "g3[a] = orc_wrap(g[a] + s1 * g1[a] + s2 * g2[a], p->grid[a]);\n  return orc_idx(p, g3);",
     "g3[a] = orc_wrap(g[a] + s1 * g1[a] - s2 * g2[a], p->grid[a]);\n  return orc_idx(p, g3);", BRUTE),
    ("phase-sign-of-the-fourth-leg", "s2 * k2[c] * rk[c] - k3[c] * rl[c]", "s2 * k2[c] * rk[c] + k3[c] * rl[c]", BRUTE),
    ("phase-without-the-sign-of-q'", "ang += s1 * k1[c] * rj[c] + s2", "ang += k1[c] * rj[c] + s2", BRUTE),
    ("phase-with-the-wrong-cell", "orc_rcart(p, ix + 7, rk);", "orc_rcart(p, ix + 4, rk);", BRUTE),
    ("fourth-leg-not-conjugated", "cplx ed = conj(orc_e(p, q3, j3, d));", "cplx ed = orc_e(p, q3, j3, d);", BRUTE),
    ("second-leg-not-conjugated", "if (s1 < 0) eb = conj(eb);\n      for (int c = 0; c < nb; ++c) {",
     "for (int c = 0; c < nb; ++c) {", BRUTE),
    ("third-leg-not-conjugated", "if (s2 < 0) ec = conj(ec);", "", BRUTE),
    ("masses-not-square-rooted", "double msq = sqrt(p->mass[ix[0]] * p->mass[ix[1]] * p->mass[ix[2]] * p->mass[ix[3]]);",
     "double msq = p->mass[ix[0]] * p->mass[ix[1]] * p->mass[ix[2]] * p->mass[ix[3]];", BRUTE),
    ("phi4-cartesian-indices-transposed", "fc[((al * 3 + be) * 3 + ga) * 3 + th]", "fc[((be * 3 + al) * 3 + ga) * 3 + th]", BRUTE),
    ("phi4-atom-legs-swapped", "b = 3 * ix[1] + be, c = 3 * ix[2] + ga, d", "b = 3 * ix[2] + be, c = 3 * ix[1] + ga, d", BRUTE),
    # three-phonon rates (Eqs. 3phgamma and V3)
    ("rates3-bose-forms-swapped", "const double B = (pr == 0) ? (n1 - n2) : (n1 + n2 + 1.0);",
     "const double B = (pr == 0) ? (n1 + n2 + 1.0) : (n1 - n2);", [RATES3]),
    ("rates3-minus-multiplicity-1", "const double mult = (pr == 0) ? 1.0 : 0.5;", "const double mult = 1.0;", [RATES3]),
    ("rates3-prefactor-1/8", "M_PI * ORC_HBAR * conv * conv * conv / (4.0 * (double)nq)",
     "M_PI * ORC_HBAR * conv * conv * conv / (8.0 * (double)nq)", [RATES3]),
    ("v3-phase-sign-of-the-third-leg", "ang += s1 * k1[c] * rj[c] - k2[c] * rk[c];",
     "ang += s1 * k1[c] * rj[c] + k2[c] * rk[c];", [RATES3]),
    ("v3-third-leg-not-conjugated", "ea * eb * conj(orc_e(p, q2, j2, c));", "ea * eb * orc_e(p, q2, j2, c);", [RATES3]),
    ("rates3-sigma-at-the-mode", "orc_sigma(&P, vel + 3 * (q1 * nb + j1), vel + 3 * (q2 * nb + j2), scalebroad, dq, dq_mode);",
     "orc_sigma(&P, vel + 3 * (q * nb + j), vel + 3 * (q2 * nb + j2), scalebroad, dq, dq_mode);", [RATES3]),
    ("rates3-gaussian-without-sqrt-pi",
     "(sqrt(M_PI) * sigma);\n              double v2 = 1.0;\n              if (!unit_vertex) {\n                if (!have_phi) {\n"
     "                  orc_phi3",
     "(sigma);\n              double v2 = 1.0;\n              if (!unit_vertex) {\n                if (!have_phi) {\n"
     "                  orc_phi3", [RATES3]),
    # three-phonon-like phase space P3 / WP3
    ("phase3-gaussian-normalised-by-sigma-squared",
     "(sqrt(M_PI) * sigma);\n            acc_p += (sgn > 0 ? 1.0 : 0.5) * delta;",
     "(sqrt(M_PI) * sigma * sigma);\n            acc_p += (sgn > 0 ? 1.0 : 0.5) * delta;", [PHASE3, RATES3]),
    ("phase3-minus-weight-1", "acc_p += (sgn > 0 ? 1.0 : 0.5) * delta;", "acc_p += delta;", [PHASE3]),
    ("phase3-wp3-plus-weight", "const double B = (sgn > 0) ? (n1 - n2) : 0.5 * (n1 + n2 + 1.0);",
     "const double B = (sgn > 0) ? (n1 + n2) : 0.5 * (n1 + n2 + 1.0);", [PHASE3]),
    # normal / Umklapp classification (reading of Sec. 2.2)
    ("umklapp-ties-to-the-largest-shift", "if (best < 0.0 || k2 < best * (1.0 - 1e-9)) {",
     "if (best < 0.0 || k2 <= best * (1.0 + 1e-9)) {", UMKLAPP),
    ("umklapp-sign-of-q'''", "- (g3[a] - n * m3[a]);", "+ (g3[a] - n * m3[a]);", UMKLAPP),
    ("umklapp-shifts-only-up-to-1",
     "  for (int m0 = -2; m0 <= 2; ++m0)\n    for (int m1 = -2; m1 <= 2; ++m1)\n      for (int m2 = -2; m2 <= 2; ++m2) {",
     "  for (int m0 = -1; m0 <= 1; ++m0)\n    for (int m1 = -1; m1 <= 1; ++m1)\n      for (int m2 = -1; m2 <= 1; ++m2) {",
     UMKLAPP),
    # a partner of zero frequency kept (reading: such terms are skipped)
    ("zero-frequency-partner-kept", "if (w3 == 0.0) continue;", "", [RATES]),
]

# (name, file under oracle/, text, replacement, pins): each text occurs exactly once in its file
PY_MUTANTS = [
    ("modes-phase-sign", "modes.py", "np.exp(2j * np.pi * float(np.dot(gfrac, R)))",
     "np.exp(-2j * np.pi * float(np.dot(gfrac, R)))", [MODES]),
    ("modes-mass-of-one-atom", "modes.py", "val.reshape(3, 3) / np.sqrt(cryst.mass[i] * cryst.mass[j])",
     "val.reshape(3, 3) / cryst.mass[i]", [MODES]),
    ("modes-velocity-without-1/2", "modes.py", "CONV * avg / (2.0 * w[k])", "CONV * avg / w[k]", [MODES]),
    ("modes-partner-not-conjugated", "modes.py", "w, U.T.conj(), -v", "w, U.T, -v", [MODES]),
    ("modes-partner-velocity-not-negated", "modes.py", "w, U.T.conj(), -v", "w, U.T.conj(), v", [MODES]),
    ("modes-eigenvectors-as-rows-not-columns", "modes.py", "om[q], ev[q], ve[q] = w, U.T, v",
     "om[q], ev[q], ve[q] = w, U, v", [MODES]),
    ("modes-velocities-not-averaged-over-degenerate-sets", "modes.py",
     "v[k] = 0.0 if w[k] == 0.0 else CONV * avg / (2.0 * w[k])",
     "v[k] = 0.0 if w[k] == 0.0 else CONV * raw[k] / (2.0 * w[k])", [MODES, RATES]),
    ("modes-gamma-acoustic-not-zeroed", "modes.py", "if q == 0 and b < 3:", "if False:", [MODES, RATES]),
    ("modes-unit-conversion-off-by-ten", "modes.py", "CONV = ECHARGE / AMU * 1e20 * 1e-24",
     "CONV = ECHARGE / AMU * 1e20 * 1e-23", [MODES]),
    ("kappa-heat-capacity-without-x", "__init__.py", "c = x * x * np.exp(x) / np.expm1(x) ** 2",
     "c = x * np.exp(x) / np.expm1(x) ** 2", [KAPPA]),
    ("kappa-without-the-cell-volume", "__init__.py", "/ (N * V)", "/ N", [KAPPA]),
    ("mlp-tanh-derivative", "mlp.py", "d3 = np.outer(dy, w4) * (1.0 - h3 * h3)", "d3 = np.outer(dy, w4) * (1.0 - h3)",
     [MLP]),
    ("mlp-loss-derivative-without-2", "mlp.py", "dy = 2.0 * r / B", "dy = r / B", [MLP]),
    ("mlp-adam-without-bias-correction", "mlp.py", "mhat = m / (1.0 - beta1 ** step)", "mhat = m", [MLP]),
]


def _union(cases):
    return sorted({p for case in cases for p in case[-1]})


def _build(src_text, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    so = os.path.join(out_dir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           "-fno-fast-math", "-D_GNU_SOURCE", "-o", so, c, "-lm"])
    return so


def _run_pins(so, pins, cwd=ROOT):
    env = dict(os.environ, FP_ORACLE_LIB=so, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        *pins], cwd=cwd, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


def _source():
    with open(SRC) as f:
        return f.read()


@pytest.fixture(scope="module")
def control_lib(tmp_path_factory):
    return _build(_source(), str(tmp_path_factory.mktemp("control")), "control")


def _tree(dst, file=None, old=None, new=None):
    """A scratch copy of the tests, the oracle package and the input generators, with one slip planted."""
    ign = shutil.ignore_patterns("__pycache__", "_build", "*.so")
    shutil.copytree(os.path.join(ROOT, "tests"), os.path.join(dst, "tests"), ignore=ign)
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"), ignore=ign)
    pkg = os.path.join(dst, "paper_2104_04895_gb300")
    os.makedirs(pkg)
    for f in os.listdir(os.path.join(ROOT, "paper_2104_04895_gb300")):
        if f.endswith(".py"):
            shutil.copy(os.path.join(ROOT, "paper_2104_04895_gb300", f), pkg)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), dst)
    if file is not None:
        path = os.path.join(dst, "oracle", file)
        with open(path) as f:
            text = f.read()
        assert text.count(old) == 1, f"{file} no longer contains the text this case mutates exactly once"
        with open(path, "w") as f:
            f.write(text.replace(old, new))
    return dst


def test_control_build_passes_the_pins(control_lib):
    rc, out = _run_pins(control_lib, _union(MUTANTS + C_MUTANTS))
    assert rc == 0, out


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(tmp_path, name, old, new, pins):
    text = _source()
    assert old in text, "the oracle no longer contains the text this case mutates"
    mutated = text.replace(old, new, 1)
    rc, out = _run_pins(_build(mutated, str(tmp_path), "mutant"), pins)
    assert rc == 1, f"{name}: the pins did not fail (pytest rc {rc})\n{out}"


@pytest.mark.parametrize("name,old,new,pins", C_MUTANTS, ids=[m[0] for m in C_MUTANTS])
def test_pins_catch_the_c_mutant(tmp_path, name, old, new, pins):
    text = _source()
    assert text.count(old) == 1, "the oracle no longer contains the text this case mutates exactly once"
    rc, out = _run_pins(_build(text.replace(old, new), str(tmp_path), "mutant"), pins)
    assert rc == 1, f"{name}: the pins did not fail (pytest rc {rc})\n{out}"


def test_control_tree_passes_the_python_pins(tmp_path, control_lib):
    rc, out = _run_pins(control_lib, _union(PY_MUTANTS), cwd=_tree(str(tmp_path / "tree")))
    assert rc == 0, out


@pytest.mark.parametrize("name,file,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_the_python_mutant(tmp_path, control_lib, name, file, old, new, pins):
    rc, out = _run_pins(control_lib, pins, cwd=_tree(str(tmp_path / "tree"), file, old, new))
    assert rc == 1, f"{name}: the pins did not fail (pytest rc {rc})\n{out}"
