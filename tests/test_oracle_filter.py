"""Pins of the oracle's matched filter (CPU).

eq:matchedfilter and the per-chunk loop (Sec. "Matched filtering") are pinned
by what the mathematics fixes independently of the oracle's own code:
* sigma^2 against the continuum integral 4 int f^(-7/3)/S df (adaptive
  quadrature plus Euler-Maclaurin end corrections);
* a noise-free injection of a bank member at SNR A is recovered with rho = A
  at exactly its sample, and no other template exceeds it (Cauchy-Schwarz);
* in Gaussian noise rho^2 is chi^2 with 2 degrees of freedom (mean 2,
  exponential tail), which fixes the data normalisation;
* the two real polarisation correlators of the paper add in quadrature to
  |z| (steps 2-3 of the per-chunk loop);
* invariances: time shift, template phase, amplitude and (d, S) scaling;
* the peak / trigger reduction on hand-built inputs with known answers.
"""

import math

import numpy as np
import pytest
from scipy import integrate, signal, stats

import oracle
import synth

N, FS, F_LOW = 1 << 16, 4096.0, 40.0


def _setup(m1=1.6, m2=2.7, pn=4):
    psd = synth.psd_onesided(N, FS)
    h, k_lo, k_hi = oracle.spa_template(m1, m2, pn, F_LOW, FS, N)
    s2 = oracle.sigma2(h, psd, FS, N, k_lo, k_hi)
    return psd, h, k_lo, k_hi, s2


def test_sigma2_matches_continuum_integral():
    for m1, m2, n in [(1.6, 2.7, N), (10.0, 10.0, N), (1.0, 1.0, 1 << 18)]:
        psd = synth.psd_onesided(n, FS)
        h, k_lo, k_hi = oracle.spa_template(m1, m2, 7, F_LOW, FS, n)
        s2 = oracle.sigma2(h, psd, FS, n, k_lo, k_hi)
        df = FS / n
        g = lambda f: f ** (-7.0 / 3.0) / float(synth.psd_analytic(f))
        a, b = k_lo * df, k_hi * df
        brk = [x for x in (60.0, 100.0, 200.0, 500.0, 1000.0) if a < x < b]
        val, _ = integrate.quad(g, a, b, points=brk or None, limit=500, epsabs=0, epsrel=1e-12)
        # sum_{k=lo}^{hi-1} g(k df) df = int_a^b g - df/2 (g(b) - g(a)) + df^2/12 (g'(b) - g'(a)) + ...
        gp = lambda f: (g(f * (1 + 1e-6)) - g(f * (1 - 1e-6))) / (2e-6 * f)
        em = val - df / 2 * (g(b) - g(a)) + df * df / 12 * (gp(b) - gp(a))
        assert abs(s2 / (4.0 * em) - 1.0) < 1e-7


@pytest.mark.parametrize("j0", [0, 1, 12345, N - 1])
def test_noise_free_injection_recovers_snr(j0):
    psd, h, k_lo, k_hi, s2 = _setup()
    d = np.zeros(N // 2 + 1, complex)
    synth.add_signal(d, h, 12.0 / math.sqrt(s2), j0, N)
    z = oracle.correlate(d, h, psd, FS, N, k_lo, k_hi)
    r = oracle.peak_triggers(z, s2, 0, N, 4096, 6.0)
    assert r["peak_j"] == j0
    assert abs(r["peak_rho"] - 12.0) < 1e-10
    # the matched template's correlator at j0 is real and positive
    assert abs(r["peak_phase"]) < 1e-10


def test_injection_is_the_maximum_over_the_bank():
    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    m1, m2 = w.masses()
    psd = w.psd()
    h, k_lo, k_hi = oracle.spa_template(m1[3], m2[3], w.pn_x2, w.f_low, w.fs, w.n)
    s2 = oracle.sigma2(h, psd, w.fs, w.n, k_lo, k_hi)
    d = np.zeros(w.n // 2 + 1, complex)
    synth.add_signal(d, h, 12.0 / math.sqrt(s2), 777, w.n)
    res = oracle.filter_bank(d, psd, m1[:16], m2[:16], w.pn_x2, w.f_low, w.fs, w.n)
    rho = np.array([r["peak_rho"] for r in res])
    assert abs(rho[3] - 12.0) < 1e-10 and res[3]["peak_j"] == 777
    assert np.all(rho <= 12.0 * (1 + 1e-12))


def test_noise_only_rho2_is_chi2_two_dof():
    psd, h, k_lo, k_hi, s2 = _setup()
    vals = []
    for seg in range(24):
        d = synth.noise_spectrum(99, seg, N, FS, psd, F_LOW)
        z = oracle.correlate(d, h, psd, FS, N, k_lo, k_hi)
        vals.append(np.abs(z[::256]) ** 2 / s2)  # decimate well beyond the correlation length
    r2 = np.concatenate(vals)
    se = np.std(r2) / math.sqrt(len(r2))
    assert abs(r2.mean() - 2.0) < 5 * se
    assert stats.kstest(r2 / 2.0, "expon").pvalue > 1e-3


def test_synthetic_noise_has_the_requested_psd():
    # Welch estimate of the coloured noise against S(f) in the band
    psd = synth.psd_onesided(N, FS)
    ests = []
    for seg in range(8):
        d = synth.strain_from_spectrum(synth.noise_spectrum(5, seg, N, FS, psd, F_LOW), N, FS)
        f, p = signal.welch(d, fs=FS, nperseg=4096, detrend=False)
        ests.append(p)
    p = np.mean(ests, axis=0)
    sel = (f > 80) & (f < 1800)
    ratio = p[sel] / synth.psd_analytic(f[sel])
    assert abs(np.median(ratio) - 1.0) < 0.03
    assert np.all(np.abs(ratio - 1.0) < 0.35)


def test_two_polarisations_add_in_quadrature():
    psd, h, k_lo, k_hi, s2 = _setup()
    d = synth.noise_spectrum(3, 0, N, FS, psd, F_LOW)
    synth.add_signal(d, h, 9.0 / math.sqrt(s2), 4000, N)
    z = oracle.correlate(d, h, psd, FS, N, k_lo, k_hi)
    cp, cx = oracle.correlate_polarisations(d, h, psd, FS, N, k_lo, k_hi)
    scale = np.max(np.abs(z))
    assert np.max(np.abs(cp - z.real)) < 1e-12 * scale
    assert np.max(np.abs(cx - z.imag)) < 1e-12 * scale
    rho = np.sqrt(cp**2 + cx**2) / math.sqrt(s2)
    assert np.max(np.abs(rho - np.abs(z) / math.sqrt(s2))) < 1e-12 * np.max(rho)


def test_invariances():
    psd, h, k_lo, k_hi, s2 = _setup()
    d = synth.noise_spectrum(4, 0, N, FS, psd, F_LOW)
    synth.add_signal(d, h, 10.0 / math.sqrt(s2), 20000, N)
    z = oracle.correlate(d, h, psd, FS, N, k_lo, k_hi)
    rho = np.abs(z) / math.sqrt(s2)
    # template phase
    z2 = oracle.correlate(d, h * np.exp(0.7j), psd, FS, N, k_lo, k_hi)
    assert np.max(np.abs(np.abs(z2) - np.abs(z))) < 1e-12 * np.max(np.abs(z))
    # template amplitude (sigma scales with it)
    z3 = oracle.correlate(d, 3.0 * h, psd, FS, N, k_lo, k_hi)
    s3 = oracle.sigma2(3.0 * h, psd, FS, N, k_lo, k_hi)
    assert np.max(np.abs(np.abs(z3) / math.sqrt(s3) - rho)) < 1e-12 * np.max(rho)
    # (d, S) -> (a d, a^2 S)
    a = 1e-3
    z4 = oracle.correlate(a * d, h, a * a * psd, FS, N, k_lo, k_hi)
    s4 = oracle.sigma2(h, a * a * psd, FS, N, k_lo, k_hi)
    assert np.max(np.abs(np.abs(z4) / math.sqrt(s4) - rho)) < 1e-10 * np.max(rho)
    # time shift of the data by s samples shifts rho by s
    s = 777
    k = np.arange(N // 2 + 1)
    d5 = d * np.exp(-2j * np.pi * ((k * s) % N) / N)
    z5 = oracle.correlate(d5, h, psd, FS, N, k_lo, k_hi)
    assert np.max(np.abs(np.abs(z5) - np.roll(np.abs(z), s))) < 1e-12 * np.max(np.abs(z))


def test_peak_and_triggers_on_known_inputs():
    n = 40
    r2 = np.zeros(n)
    r2[3], r2[5] = 50.0, 50.0      # tie in window 0 -> lowest j (3)
    r2[12] = 30.0                  # window 1 below threshold 6 (36)
    r2[20], r2[27] = 64.0, 81.0    # window 2: max at 27
    r2[33] = 81.0                  # window 3 ties window 2's maximum -> peak stays at 27
    units = np.array([1, 1j, -1, -1j])  # exact unit phases keep the planted ties exact
    z = np.sqrt(r2) * units[np.arange(n) % 4]
    r = oracle.peak_triggers(z, 1.0, 0, n, 10, 6.0)
    assert r["peak_j"] == 27 and abs(r["peak_rho"] - 9.0) < 1e-15
    assert list(r["trig_j"]) == [3, 27, 33]
    assert np.allclose(r["trig_rho"], [math.sqrt(50), 9, 9])
    assert np.allclose(r["trig_phase"], np.angle(z[[3, 27, 33]]))
    # valid range and a ragged last window: [5, 34) -> windows [5,15) [15,25) [25,34)
    r = oracle.peak_triggers(z, 1.0, 5, 34, 10, 6.0)
    assert list(r["trig_j"]) == [5, 20, 27]
    assert r["peak_j"] == 27
    # threshold is strict: rho == thr is not a trigger
    r = oracle.peak_triggers(z, 1.0, 0, n, 10, 9.0)
    assert r["n_trig"] == 0
    # all-zero correlator and sigma2 == 0: rho = 0, peak at the first valid sample
    r = oracle.peak_triggers(np.zeros(n, complex), 0.0, 7, n, 10, 6.0)
    assert r["peak_j"] == 7 and r["peak_rho"] == 0.0 and r["n_trig"] == 0


def test_filter_template_composes_the_steps():
    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    m1, m2 = w.masses()
    psd = w.psd()
    d = w.noise()
    r = oracle.filter_template(d, psd, m1[0], m2[0], w.pn_x2, w.f_low, w.fs, w.n, thr=4.0)
    h, k_lo, k_hi = oracle.spa_template(m1[0], m2[0], w.pn_x2, w.f_low, w.fs, w.n)
    s2 = oracle.sigma2(h, psd, w.fs, w.n, k_lo, k_hi)
    z = oracle.correlate(d, h, psd, w.fs, w.n, k_lo, k_hi)
    r2 = oracle.peak_triggers(z, s2, 0, w.n, int(w.fs), 4.0)
    assert r["sigma2"] == s2
    assert r["peak_j"] == r2["peak_j"] and r["peak_rho"] == r2["peak_rho"]
    assert list(r["trig_j"]) == list(r2["trig_j"])
