"""Pins of the oracle's multi-band functions (host only): the direct-sum band
correlator against the FFT route at sample times and, between samples, against
the FFT route of a zero-padded spectrum; the band edges on single bins; bands
adding up; the exact band SNR of a bank-member injection; the band-limited
filter; the same sums from a decimated copy of the segment; and the
band-limited, resampled series on sums of cosines."""

import math

import numpy as np
import pytest

import oracle
import synth

N, FS, F_LOW = 1 << 13, 4096.0, 30.0  # df = 0.5 Hz: the 4 df factor is not 1
M1, M2, PN = 3.0, 2.0, 7
DF = FS / N


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


@pytest.fixture(scope="module")
def noisy():
    psd = synth.psd_onesided(N, FS)
    d = synth.noise_spectrum(11, 0, N, FS, psd, F_LOW)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    synth.add_signal(d, h, 9.0 / math.sqrt(oracle.sigma2(h, psd, FS, N, lo, hi)), 5000, N)
    return d, psd


def test_full_band_direct_sums_equal_the_fft_route(noisy):
    d, psd = noisy
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    zf = oracle.correlate(d, h, psd, FS, N, lo, hi)
    js = [0, 1, 777, 5000, 8000, N - 1]
    z, s2 = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, [j / FS for j in js], 0.0, 0.0)
    assert np.max(np.abs(z - zf[js])) < 1e-9 * np.max(np.abs(zf))
    assert abs(s2 - oracle.sigma2(h, psd, FS, N, lo, hi)) < 1e-12 * s2


def test_between_samples_equals_the_upsampled_fft_route(noisy):
    # t = (j + 1/2) / fs is sample 2j + 1 of the same spectrum at twice the
    # rate (same df, zero bins above fs/2): an independent route
    d, psd = noisy
    n2 = 2 * N
    d2 = np.zeros(n2 // 2 + 1, dtype=np.complex128)
    d2[: N // 2 + 1] = d
    psd2 = np.ones(n2 // 2 + 1)
    psd2[: N // 2 + 1] = psd
    psd2[0] = 1.0
    h2, lo2, hi2 = oracle.spa_template(M1, M2, PN, F_LOW, 2 * FS, n2)
    zf = oracle.correlate(d2, h2, psd2, 2 * FS, n2, lo2, hi2)
    js = [3, 4999, 8000]
    z, _ = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, [(j + 0.5) / FS for j in js], 0.0, 0.0)
    assert np.max(np.abs(z - zf[[2 * j + 1 for j in js]])) < 1e-9 * np.max(np.abs(zf))


def test_single_bin_edges_and_time_dependence():
    psd = synth.psd_onesided(N, FS)
    k0 = 1000  # 500 Hz, inside the template's band
    d = np.zeros(N // 2 + 1, dtype=np.complex128)
    d[k0] = 1.0 + 0.5j
    f0 = k0 * DF
    eps = 1e-6
    t = [0.0, 0.3217, 1.7]
    z_in, s_in = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, f0, f0 + DF)
    assert np.all(np.abs(z_in) > 0) and s_in > 0
    # |z| is constant and the phase turns at f0
    assert np.max(np.abs(np.abs(z_in) - abs(z_in[0]))) < 1e-12 * abs(z_in[0])
    for i in (1, 2):
        assert abs(z_in[i] - z_in[0] * np.exp(2j * math.pi * f0 * t[i])) < 1e-9 * abs(z_in[0])
    # f_lo inclusive, f_hi exclusive
    for lo, hi in ((f0 + eps, 0.0), (F_LOW, f0), (f0 - DF, f0 - eps)):
        z, s = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, lo, hi)
        assert np.all(z == 0)
    z, _ = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, F_LOW, f0 + eps)
    assert np.max(np.abs(z - z_in)) < 1e-15 * abs(z_in[0])


def test_bands_add_up(noisy):
    d, psd = noisy
    t = [0.1, 1.2207031, 3.0]
    zs, ss = zip(*[oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, a, b)
                   for a, b in ((0.0, 60.0), (60.0, 150.0), (150.0, 0.0))])
    zf, sf = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, 0.0, 0.0)
    assert np.max(np.abs(sum(zs) - zf)) < 1e-12 * np.max(np.abs(zf))
    assert abs(sum(ss) - sf) < 1e-12 * sf
    assert all(s > 0 for s in ss)


def test_band_snr_of_an_exact_injection():
    # a noise-free bank member of SNR A sigma: in every band B, z_B(j0) =
    # A sigma_B^2 (real), so rho_B = SNR sigma_B / sigma (Cauchy-Schwarz equality)
    psd = synth.psd_onesided(N, FS)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    s2 = oracle.sigma2(h, psd, FS, N, lo, hi)
    d = np.zeros(N // 2 + 1, dtype=np.complex128)
    j0 = 4321
    synth.add_signal(d, h, 12.0 / math.sqrt(s2), j0, N)
    for a, b in ((0.0, 0.0), (0.0, 80.0), (80.0, 0.0), (45.0, 200.0)):
        z, sb = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, [j0 / FS], a, b)
        assert abs(abs(z[0]) / math.sqrt(sb) - 12.0 * math.sqrt(sb / s2)) < 1e-9
        assert abs(z[0].imag) < 1e-9 * abs(z[0])


def test_band_filter(noisy):
    d, psd = noisy
    full = oracle.filter_template(d, psd, M1, M2, PN, F_LOW, FS, N)
    same = oracle.band_filter_template(d, psd, M1, M2, PN, F_LOW, FS, N, 0.0, 0.0)
    assert same["peak_j"] == full["peak_j"] and abs(same["peak_rho"] - full["peak_rho"]) < 1e-12
    assert abs(same["sigma2"] - full["sigma2"]) < 1e-12 * full["sigma2"]
    assert np.array_equal(same["trig_j"], full["trig_j"])
    hb = oracle.band_filter_template(d, psd, M1, M2, PN, F_LOW, FS, N, 70.0, 400.0)
    z, sb = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, [hb["peak_j"] / FS], 70.0, 400.0)
    assert abs(sb - hb["sigma2"]) < 1e-12 * sb
    assert abs(abs(z[0]) / math.sqrt(sb) - hb["peak_rho"]) < 1e-9 * hb["peak_rho"]
    assert abs(hb["peak_j"] - 5000) <= 2


def test_decimated_segment_gives_the_same_band_sums(noisy):
    # the same data at a quarter of the rate: the first N/8 bins, the same df;
    # a band below the new Nyquist frequency sums the same terms
    d, psd = noisy
    n4, fs4 = N // 4, FS / 4
    d4 = d[: n4 // 2 + 1].copy()
    d4[-1] = 0.0
    psd4 = psd[: n4 // 2 + 1]
    t = [0.0, 0.75, 2.5]
    z, s = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, t, 0.0, 400.0)
    z4, s4 = oracle.band_correlate(d4, psd4, M1, M2, PN, F_LOW, fs4, n4, t, 0.0, 400.0)
    assert np.max(np.abs(z4 - z)) < 1e-12 * np.max(np.abs(z))
    assert abs(s4 - s) < 1e-12 * s


def test_band_series_keeps_the_band_and_decimates():
    # three cosines, at bins 100 (below the band), 900 (in it) and 1900
    # (above it, and above the Nyquist frequency of the decimated rate)
    n, fs = 1 << 12, 4096.0
    j = np.arange(n)
    comp = {k: a * np.cos(2 * math.pi * k * j / n + p) for k, a, p in ((100, 1.0, 0.3), (900, 0.7, 1.1),
                                                                       (1900, 0.4, -0.5))}
    x = sum(comp.values())
    df = fs / n
    for decim in (1, 2):
        y = oracle.band_series(x, fs, 500 * df, 1500 * df, decim)
        want = comp[900][::decim]
        assert len(y) == n // decim
        assert np.max(np.abs(y - want)) < 1e-12
    # the full band at the full rate gives the strain back (no Nyquist content)
    assert np.max(np.abs(oracle.band_series(x, fs, 0.0, 0.0, 1) - x)) < 1e-12
    # edges: a band starting exactly at bin 900 keeps it, one just above drops it
    assert np.max(np.abs(oracle.band_series(x, fs, 900 * df, 901 * df, 1) - comp[900])) < 1e-12
    assert np.max(np.abs(oracle.band_series(x, fs, 900 * df + 1e-9, 1500 * df, 1))) < 1e-12
