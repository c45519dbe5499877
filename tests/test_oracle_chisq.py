"""Pins of the oracle's chi^2 signal-consistency test (host only): zero for a
single band, ~0 for the exact template, the band sums adding up to the full
correlator, and the chi-squared mean 2p - 2 in Gaussian noise."""

import math

import numpy as np
import pytest

import oracle
import synth

N, FS, F_LOW = 1 << 13, 4096.0, 30.0  # df = 0.5 Hz: the 4 df factor is not 1
M1, M2, PN = 3.0, 2.0, 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _injection(amp_snr, j0):
    psd = synth.psd_onesided(N, FS)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    s2 = oracle.sigma2(h, psd, FS, N, lo, hi)
    d = np.zeros(N // 2 + 1, dtype=np.complex128)
    synth.add_signal(d, h, amp_snr / math.sqrt(s2), j0, N)
    return d, psd


def test_single_band_is_zero():
    d, psd = _injection(10.0, 1234)
    chi, _ = oracle.chisq(d, psd, M1, M2, PN, F_LOW, FS, N, [1234, 77], 1)
    assert np.all(np.abs(chi) < 1e-20 * (1 + 100.0))


def test_exact_template_is_consistent():
    d, psd = _injection(10.0, 1234)
    chi, rho = oracle.chisq(d, psd, M1, M2, PN, F_LOW, FS, N, [1234], 16)
    assert abs(rho[0] - 10.0) < 1e-9
    # the bands hold equal power up to one bin each, so chi^2 << rho^2 = 100
    assert chi[0] < 1e-3 * rho[0] ** 2


def test_band_sums_give_the_correlator():
    psd = synth.psd_onesided(N, FS)
    d = synth.noise_spectrum(7, 1, N, FS, psd, F_LOW)
    samples = [0, 5, 4097, N - 1]
    _, rho = oracle.chisq(d, psd, M1, M2, PN, F_LOW, FS, N, samples, 8)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    z = oracle.correlate(d, h, psd, FS, N, lo, hi)
    s2 = oracle.sigma2(h, psd, FS, N, lo, hi)
    assert np.allclose(rho, np.abs(z[samples]) / math.sqrt(s2), rtol=1e-10)


def test_noise_mean_is_2p_minus_2():
    psd = synth.psd_onesided(N, FS)
    p = 8
    vals = []
    for seg in range(4):
        d = synth.noise_spectrum(11, seg, N, FS, psd, F_LOW)
        chi, _ = oracle.chisq(d, psd, M1, M2, PN, F_LOW, FS, N, range(0, N, 128), p)
        vals.append(chi)
    mean = np.concatenate(vals).mean()
    assert abs(mean - (2 * p - 2)) < 0.1 * (2 * p - 2), mean
