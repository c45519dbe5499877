"""The oracle's pins are strong enough: plausible mistakes planted in a copy of
the oracle's C source (on the CPU, never in the library) each make the pin
suite fail.  The unmodified copy, built the same way, passes."""

import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cui_oracle.c")
PINS = ["tests/test_oracle_fft.py", "tests/test_oracle_template.py", "tests/test_oracle_filter.py"]

# (name, text in cui_oracle.c, replacement)
MUTANTS = [
    ("fft_twiddle_sign", "double a = sign * 2.0 * OR_PI * (double)m / (double)len;",
     "double a = -sign * 2.0 * OR_PI * (double)m / (double)len;"),
    ("fft_no_bit_reversal", "if (i < j) {", "if (i < 0) {"),
    ("spectrum_no_dt", "dr[k] = dt * xr[k]; di[k] = dt * xi[k];", "dr[k] = xr[k]; di[k] = xi[k];"),
    ("alpha2_sign", "a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0;", "a[2] = 3715.0 / 756.0 - 55.0 * eta / 9.0;"),
    ("alpha3_sign", "a[3] = -16.0 * pi;", "a[3] = 16.0 * pi;"),
    ("alpha4_digit", "27145.0 * eta / 504.0", "27154.0 * eta / 504.0"),
    ("alpha5_log_factor", "(1.0 + 3.0 * log(v / v_lso))", "(1.0 + 2.0 * log(v / v_lso))"),
    ("alpha6_log", "- 6848.0 / 21.0 * log(4.0 * v);", "- 6848.0 / 21.0 * log(v);"),
    ("alpha7_digit", "378515.0 * eta / 1512.0", "378155.0 * eta / 1512.0"),
    ("newtonian_power", "double v5 = v * v * v * v * v;", "double v5 = v * v * v * v;"),
    ("mass_constant", "#define OR_MSUN_S 4.925490947e-6", "#define OR_MSUN_S 4.952490947e-6"),
    ("amplitude_power", "pow(f[k - lo], -7.0 / 6.0)", "pow(f[k - lo], -7.0 / 3.0)"),
    ("template_phase_sign", "hi[k] = -amp * sin(psi[k - lo]);", "hi[k] = amp * sin(psi[k - lo]);"),
    ("band_floor", "long lo = (long)ceil(f_low / df);", "long lo = (long)floor(f_low / df);"),
    ("isco_power", "pow(6.0, 1.5)", "pow(6.0, 0.5)"),
    ("sigma_factor", "return 4.0 * df * s;", "return 2.0 * df * s;"),
    ("correlate_no_conj", "zr[k] = (dr[k] * hr[k] + di[k] * hi[k]) / psd[k];\n        zi[k] = (di[k] * hr[k] - dr[k] * hi[k]) / psd[k];",
     "zr[k] = (dr[k] * hr[k] - di[k] * hi[k]) / psd[k];\n        zi[k] = (di[k] * hr[k] + dr[k] * hi[k]) / psd[k];"),
    ("correlate_no_psd", "zi[k] = (di[k] * hr[k] - dr[k] * hi[k]) / psd[k];", "zi[k] = (di[k] * hr[k] - dr[k] * hi[k]);"),
    ("correlate_sign", "if (or_fft(n, +1, zr, zi) != 0) return -1;", "if (or_fft(n, -1, zr, zi) != 0) return -1;"),
    ("correlate_factor", "zr[j] *= 4.0 * df; zi[j] *= 4.0 * df;", "zr[j] *= 2.0 * df; zi[j] *= 2.0 * df;"),
    ("cross_polarisation_sign", "double ti = pol == 0 ? hi[k] : hr[k];", "double ti = pol == 0 ? hi[k] : -hr[k];"),
    ("peak_ties_high", "if (r2 > wbest) { wbest = r2; wj = j; }", "if (r2 >= wbest) { wbest = r2; wj = j; }"),
    ("threshold_not_strict", "if (sqrt(wbest) > thr) {", "if (sqrt(wbest) >= thr) {"),
    ("window_overlap", "for (long w0 = lo; w0 < hi; w0 += window) {", "for (long w0 = lo; w0 < hi; w0 += window - 1) {"),
]


def _build(tmp_path, name, text):
    c = tmp_path / f"{name}.c"
    c.write_text(text)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"])
    return str(so)


def _pins_pass(so):
    env = dict(os.environ, CUI_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode == 0


def test_unmodified_copy_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "control", open(SRC).read()))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    assert not _pins_pass(_build(tmp_path, name, src.replace(old, new)))
