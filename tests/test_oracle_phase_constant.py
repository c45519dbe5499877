"""The absolute constant of the TaylorF2 phase, pinned by a direct Fourier
transform (CPU).

The stationary-phase approximation gives the phase of a chirp's Fourier
transform up to a constant and a term linear in f, and the second-derivative
pin (d^2 Psi / df^2 from the binding energy and flux) is blind to both.  Here
the oracle's own time-domain chirp (TaylorT2, t_c = phi_c = 0, the chirp
coalescing at sample 0) is transformed with numpy's FFT, and the phase of
H(f) = dt sum_j h_+(t_j) e^{-2 pi i f t_j} at mid-band is compared with
-Psi_F2(f) of the frequency-domain oracle.  For a real chirp h_+ = A cos 2 phi
with increasing frequency the stationary point of e^{i(2 phi - 2 pi f t)}
contributes e^{+i pi/4}, so arg H = -(2 pi f t_f - 2 phi(t_f) - pi/4):

* below 2.5PN the offset arg H + Psi_F2 must be 0 (a missing -pi/4 would read
  0.79 rad, a flipped sign of the template phase a slope in f);
* at 2.5PN the frequency-domain logarithm is referred to v_lso = 6^(-1/2)
  (the "1 + 3 ln(v / v_lso)" of the TaylorF2 literature) while the
  time-domain phase integrates ln v from phi_c = 0.  Carrying the 2.5PN terms
  of t(v) and phi(v) through Psi = 2 pi f t - 2 phi - pi/4 (the v^5 term of t
  gives the constant -10 a_5 / (96 eta), of phi the log) and comparing with
  (3 / (128 eta)) alpha_5 (1 + 3 ln(v / v_lso)) leaves the constant
  9 alpha_5 ln 6 / (256 eta), alpha_5 = pi (38645/756 - 65 eta / 9), which the
  offset must equal (mod 2 pi).  Terms beyond 2.5PN add powers of v, no
  constant.

The chirps fit inside the segment and the comparison skips the band edges,
where the abrupt start and end of the time-domain waveform ring."""

import math

import numpy as np
import pytest

import oracle
from oracle import td


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def offsets(m1, m2, pn, f_low, fs=4096.0, n=1 << 16):
    M = (m1 + m2) * td.MSUN_S
    hp, _ = td.td_template(m1, m2, pn, f_low, fs, n)
    H = np.fft.rfft(hp) / fs
    f = np.arange(n // 2 + 1) * fs / n
    sel = (f > 1.6 * f_low) & (f < 0.6 / (6 ** 1.5 * math.pi * M))
    psi = oracle.spa_phase(m1, m2, pn, f[sel])
    return np.angle(H[sel] * np.exp(1j * psi))


def wrap(x):
    return (x + math.pi) % (2 * math.pi) - math.pi


@pytest.mark.parametrize("m1,m2,f_low", [(10.0, 10.0, 30.0), (5.0, 3.0, 40.0), (1.4, 1.4, 60.0)])
@pytest.mark.parametrize("pn", [0, 2, 3, 4])
def test_below_2p5pn_the_phase_has_no_free_constant(m1, m2, f_low, pn):
    d = offsets(m1, m2, pn, f_low)
    assert abs(np.mean(d)) < 0.02, np.mean(d)
    assert np.std(d) < 0.08, np.std(d)  # no slope: no time offset either


@pytest.mark.parametrize("m1,m2,f_low", [(10.0, 10.0, 30.0), (5.0, 3.0, 40.0), (1.4, 1.4, 60.0)])
def test_2p5pn_constant_is_the_lso_reference_of_the_log(m1, m2, f_low):
    eta = m1 * m2 / (m1 + m2) ** 2
    alpha5 = math.pi * (38645.0 / 756.0 - 65.0 * eta / 9.0)
    want = wrap(9.0 * alpha5 * math.log(6.0) / (256.0 * eta))
    d = offsets(m1, m2, 5, f_low)
    assert abs(wrap(np.mean(d) - want)) < 0.03, (np.mean(d), want)
    assert np.std(d) < 0.08


def test_the_pins_see_a_missing_quarter_turn_and_a_flipped_sign():
    """The same comparison against a phase without the -pi/4, and against the
    conjugate template, fails the bounds above."""
    m1, m2, f_low, fs, n = 10.0, 10.0, 30.0, 4096.0, 1 << 16
    M = (m1 + m2) * td.MSUN_S
    hp, _ = td.td_template(m1, m2, 2, f_low, fs, n)
    H = np.fft.rfft(hp) / fs
    f = np.arange(n // 2 + 1) * fs / n
    sel = (f > 1.6 * f_low) & (f < 0.6 / (6 ** 1.5 * math.pi * M))
    psi = oracle.spa_phase(m1, m2, 2, f[sel])
    no_quarter = np.angle(H[sel] * np.exp(1j * (psi + math.pi / 4)))
    flipped = np.angle(H[sel] * np.exp(-1j * psi))
    assert abs(np.mean(no_quarter)) > 0.5
    assert np.std(flipped) > 0.5 or abs(np.mean(flipped)) > 0.5
