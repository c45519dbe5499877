"""Pins of the prescreen oracle (CPU): features against an FFT-based
computation (numpy) and their noise expectation, the convolution against
scipy's correlate, the loss on known cases, and every gradient against central
finite differences."""

import math

import numpy as np
from scipy import signal

import synth
from oracle import prescreen as ps


def test_features_match_fft_based_band_power():
    n, fs, f_low = 1 << 12, 4096.0, 30.0
    psd = synth.psd_onesided(n, fs)
    d = synth.noise_spectrum(8, 0, n, fs, psd, f_low)
    F = ps.features(d, psd, n, fs, f_low, bands=4, frame=256)
    df = fs / n
    for b, (k0, k1) in enumerate(ps.band_edges(n, fs, f_low, 4)):
        spec = np.zeros(n, complex)
        spec[k0:k1] = d[k0:k1] * np.sqrt(4 * df / psd[k0:k1])
        x = np.fft.ifft(spec) * n
        p = (np.abs(x) ** 2).reshape(-1, 256).mean(axis=1)
        assert np.allclose(F[b], np.log(p / (2 * (k1 - k0))), atol=1e-9)


def test_features_have_unit_power_in_noise():
    n, fs, f_low = 1 << 14, 4096.0, 30.0
    psd = synth.psd_onesided(n, fs)
    vals = []
    for seg in range(6):
        d = synth.noise_spectrum(9, seg, n, fs, psd, f_low)
        vals.append(np.exp(ps.features(d, psd, n, fs, f_low, bands=8, frame=512)))
    r = np.concatenate(vals, axis=1)
    assert abs(r.mean() - 1.0) < 0.05


def test_band_edges_are_log_spaced_and_cover_the_band():
    e = ps.band_edges(1 << 16, 4096.0, 20.0, 8)
    assert e[0][0] == math.ceil(20.0 * 16) and e[-1][1] == 1 << 15
    assert all(a[1] == b[0] for a, b in zip(e, e[1:]))
    widths = np.array([k1 - k0 for k0, k1 in e], dtype=float)
    assert np.all(np.diff(np.log(widths)) > 0.5)


def test_convolution_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 20))
    W = rng.standard_normal((2, 3, 5))
    b = rng.standard_normal(2)
    for stride in (1, 2):
        out = ps._conv(x, W, b, stride)
        for o in range(2):
            full = sum(signal.correlate(np.pad(x[i], 2), W[o, i], mode="valid") for i in range(3)) + b[o]
            assert np.allclose(out[o], full[::stride])


def test_loss_on_known_cases():
    theta = np.zeros(ps.n_params())
    x = np.zeros((8, 128))
    y = ps.soft_labels(40)
    assert abs(y.sum() - 1) < 1e-15 and y[40] == 2 * y[41]
    # all-zero parameters give uniform logits: loss = log R
    assert abs(ps.loss(theta, [x], [y]) - math.log(100)) < 1e-12


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    bands, regions = 3, 7
    npar = ps.n_params(bands, regions)
    theta = rng.standard_normal(npar) * 0.3
    xs = [rng.standard_normal((bands, 32)) for _ in range(2)]
    ys = [ps.soft_labels(int(r), regions) for r in (2, 6)]
    g = ps.gradient(theta, xs, ys, bands, regions)
    idx = rng.choice(npar, 60, replace=False)
    # include every bias block and the pooled layers
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ps.loss(tp, xs, ys, bands, regions) - ps.loss(tm, xs, ys, bands, regions)) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_regions_are_equal_count_and_ordered():
    m1, m2 = synth.sample_masses(3, 1, 1000, 1.0, 25.0, True)
    groups, bounds = ps.regions_of_bank(m1, m2, 100)
    assert sorted(np.concatenate(groups).tolist()) == list(range(1000))
    assert all(len(g) == 10 for g in groups)
    mc = ps.chirp_mass(m1, m2)
    assert all(mc[g].max() <= mc[h].min() for g, h in zip(groups, groups[1:]))
    assert ps.region_of(mc[groups[37][0]], bounds) == 37
