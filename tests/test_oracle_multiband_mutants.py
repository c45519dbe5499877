"""The multi-band pins catch plausible mistakes: copies of the oracle's band
correlator and band series with one planted error each (a sign, a band edge,
a factor, a conjugate, the time scale, the decimated scaling) must fail the
same properties the oracle itself passes."""

import math

import numpy as np
import pytest

import oracle
import synth

N, FS, F_LOW = 1 << 13, 4096.0, 30.0  # df = 0.5 Hz, so a missing 4 df factor shows
M1, M2, PN = 3.0, 2.0, 7
DF = FS / N


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def correlate_variant(dtilde, psd, times, f_lo, f_hi, mistake=None):
    """The oracle's band correlator, written out again with one optional mistake."""
    h, _, _ = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    ka, kb = oracle.band_edges(M1, M2, F_LOW, FS, N, f_lo, f_hi)
    if mistake == "edge_floor":
        ka = max(ka - 1, 0)
    k = np.arange(ka, kb)
    fac = 1.0 if mistake == "no_4df" else 4.0 * DF
    hh = h[ka:kb] if mistake == "no_conj" else np.conj(h[ka:kb])
    terms = fac * np.asarray(dtilde)[ka:kb] * hh / psd[ka:kb]
    sign = -1.0 if mistake == "time_sign" else 1.0
    scale = 2.0 if mistake == "time_scale" else 1.0
    z = np.empty(len(times), dtype=np.complex128)
    for i, t in enumerate(times):
        x = (float(t) * DF * scale) % 1.0
        z[i] = np.sum(terms * np.exp(sign * 2j * math.pi * ((k * x) % 1.0)))
    return z


def series_variant(strain, f_lo, f_hi, decim, mistake=None):
    n = len(strain)
    m = n // decim
    df = FS / n
    X = oracle.segment_spectrum(strain, FS) * FS
    k = np.arange(m // 2 + 1)
    ka = int(np.ceil(f_lo / df))
    kb = m // 2 if f_hi <= 0 else min(m // 2, int(np.ceil(f_hi / df)))
    if mistake == "hi_inclusive":
        kb = min(m // 2, kb + 1)
    Y = np.where((k >= ka) & (k < kb), X[: m // 2 + 1], 0.0)
    out = np.fft.irfft(Y, m)
    return out if mistake == "decim_scale" else out * (m / n)


@pytest.fixture(scope="module")
def noisy():
    psd = synth.psd_onesided(N, FS)
    d = synth.noise_spectrum(11, 0, N, FS, psd, F_LOW)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    synth.add_signal(d, h, 9.0 / math.sqrt(oracle.sigma2(h, psd, FS, N, lo, hi)), 5000, N)
    return d, psd


def fft_route_pin(z_of, d, psd):
    """Full band at sample times equals the FFT route."""
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    zf = oracle.correlate(d, h, psd, FS, N, lo, hi)
    js = [0, 1, 777, 5000, 8000]
    z = z_of(d, psd, [j / FS for j in js], 0.0, 0.0)
    return np.max(np.abs(z - zf[js])) < 1e-9 * np.max(np.abs(zf))


def edge_pin(z_of, psd):
    """A band starting exactly at a bin holds it; one starting just above drops it."""
    k0 = 1000  # 500 Hz, inside the template's band
    d = np.zeros(N // 2 + 1, dtype=np.complex128)
    d[k0 - 1] = 1.0
    d[k0] = 1.0 + 0.5j
    z_in = z_of(d, psd, [0.3], k0 * DF, (k0 + 1) * DF)
    z_one = 4.0 * DF * d[k0] * np.conj(oracle.spa_template(M1, M2, PN, F_LOW, FS, N)[0][k0]) / psd[k0]
    z_one *= np.exp(2j * math.pi * k0 * DF * 0.3)
    return abs(z_in[0] - z_one) < 1e-12 * abs(z_one)


def test_unmodified_variant_passes(noisy):
    d, psd = noisy

    def z_of(dd, pp, t, a, b):
        return correlate_variant(dd, pp, t, a, b)

    assert fft_route_pin(z_of, d, psd)
    assert edge_pin(z_of, psd)
    z_ref, _ = oracle.band_correlate(d, psd, M1, M2, PN, F_LOW, FS, N, [0.1, 2.5], 60.0, 300.0)
    assert np.max(np.abs(z_of(d, psd, [0.1, 2.5], 60.0, 300.0) - z_ref)) < 1e-12 * np.max(np.abs(z_ref))


@pytest.mark.parametrize("mistake", ["edge_floor", "no_4df", "no_conj", "time_sign", "time_scale"])
def test_planted_correlator_mistake_is_caught(noisy, mistake):
    d, psd = noisy

    def z_of(dd, pp, t, a, b):
        return correlate_variant(dd, pp, t, a, b, mistake)

    assert not (fft_route_pin(z_of, d, psd) and edge_pin(z_of, psd)), mistake


def cosine_pin(series):
    """Cosines below, inside and above the band: only the one inside survives,
    at the full and at half the rate."""
    n = 1 << 12
    j = np.arange(n)
    df = FS / n
    comp = {k: a * np.cos(2 * math.pi * k * j / n + p) for k, a, p in ((100, 1.0, 0.3), (900, 0.7, 1.1),
                                                                       (1500, 0.4, -0.5))}
    x = sum(comp.values())
    ok = True
    for decim in (1, 2):
        y = series(x, 500 * df, 1500 * df, decim)
        ok &= len(y) == n // decim and np.max(np.abs(y - comp[900][::decim])) < 1e-12
    return bool(ok)


def test_series_variant_passes():
    assert cosine_pin(lambda x, a, b, dec: series_variant(x, a, b, dec))
    assert cosine_pin(lambda x, a, b, dec: oracle.band_series(x, FS, a, b, dec))


@pytest.mark.parametrize("mistake", ["hi_inclusive", "decim_scale"])
def test_planted_series_mistake_is_caught(mistake):
    assert not cosine_pin(lambda x, a, b, dec: series_variant(x, a, b, dec, mistake)), mistake
