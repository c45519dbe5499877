"""Seeded synthetic inputs for the bank matched filter.

This module is shared by the tests, the benchmark and the smoke check, and it
is deliberately free of the matched filter's own arithmetic: it draws random
numbers, evaluates the analytic detector noise curve the workloads are stated
with, colours Gaussian noise by that curve, samples template masses and
injection times, and adds *caller-supplied* frequency-domain signals into a
segment spectrum.  Template waveforms, their norms and every filter output
come from elsewhere (the oracle in the tests, the library in the benchmark).

Random numbers come from one counter-based generator: the SplitMix64 output
function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``key(seed, stream) + (i + 1) * gamma``,
so every draw is addressable by (seed, stream, index) and independent of the
order in which draws are made.  Normal deviates use the Box-Muller transform.

Workload recipes (sizes, mass ranges, lower cut-off, injections) are listed in
``WORKLOADS``; each is a stand-in, with synthetic Gaussian noise, for the
detector data analysed in the paper (Sec. "GPU based detection pipeline
performances and profiling").
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "GAMMA", "mix64", "uniform", "uniform_open", "normal_pairs",
    "psd_analytic", "psd_onesided", "band_start", "noise_spectrum",
    "strain_from_spectrum", "add_signal", "sample_masses",
    "injection_times", "injection_snrs", "Workload", "WORKLOADS",
]

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    t = np.uint64(stream & 0xFFFFFFFFFFFFFFFF)
    return mix64(mix64(s) ^ mix64(t + GAMMA))


def _raw(seed: int, stream: int, count: int, offset: int = 0):
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(_key(seed, stream) + idx * GAMMA)


def uniform(seed: int, stream: int, count: int, offset: int = 0):
    """Doubles in [0, 1) with 53 random bits."""
    return (_raw(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64) * 2.0**-53


def uniform_open(seed: int, stream: int, count: int, offset: int = 0):
    """Doubles in (0, 1], safe for a logarithm."""
    r = (_raw(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64)
    return (r + 1.0) * 2.0**-53


def normal_pairs(seed: int, stream: int, count: int):
    """``count`` pairs of independent standard normal deviates (Box-Muller)."""
    u1 = uniform_open(seed, stream, count, 0)
    u2 = uniform(seed, stream, count, count)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)


def psd_analytic(f, scale: float = 1.0):
    """One-sided noise PSD (1/Hz) of the analytic curve the workloads use,
    S(f) = 9e-46 [(4.49 x)^-56 + 0.16 x^-4.52 + 0.52 + 0.32 x^2], x = f/150 Hz.
    Returns +inf at f = 0."""
    f = np.asarray(f, dtype=np.float64)
    with np.errstate(divide="ignore", over="ignore"):
        x = f / 150.0
        s = 9e-46 * ((4.49 * x) ** -56 + 0.16 * x ** -4.52 + 0.52 + 0.32 * x * x)
    s = np.where(f > 0, s, np.inf)
    return s * scale


def psd_onesided(n: int, fs: float, scale: float = 1.0):
    """S_k at f_k = k fs / n for k = 0..n/2 (FP64)."""
    return psd_analytic(np.arange(n // 2 + 1) * (fs / n), scale)


def band_start(f_low: float, n: int, fs: float) -> int:
    """First one-sided bin at or above ``f_low``."""
    return int(math.ceil(f_low * n / fs))


def noise_spectrum(seed: int, stream: int, n: int, fs: float, psd, f_low: float):
    """Gaussian noise spectrum d~_k (k = 0..n/2) with E|d~_k|^2 = S_k / (2 df)
    on [f_low, fs/2) and exactly zero elsewhere (DC, below f_low, Nyquist)."""
    df = fs / n
    k0 = band_start(f_low, n, fs)
    nb = n // 2 - k0
    out = np.zeros(n // 2 + 1, dtype=np.complex128)
    if nb <= 0:
        return out
    g1, g2 = normal_pairs(seed, stream, nb)
    amp = np.sqrt(np.asarray(psd, dtype=np.float64)[k0 : n // 2] / (4.0 * df))
    out[k0 : n // 2] = amp * (g1 + 1j * g2)
    return out


def strain_from_spectrum(dtilde, n: int, fs: float):
    """Real time series d_j whose spectrum Delta t * sum_j d_j e^{-2 pi i jk/n}
    equals ``dtilde`` (numpy's inverse real FFT divided by Delta t)."""
    return np.fft.irfft(np.asarray(dtilde, dtype=np.complex128), n) * fs


def add_signal(dtilde, stilde, amplitude: float, j0: int, n: int):
    """dtilde += amplitude * stilde * exp(-2 pi i k j0 / n): a caller-supplied
    one-sided signal spectrum delayed by ``j0`` samples (circularly)."""
    k = np.arange(len(dtilde), dtype=np.int64)
    ph = ((k * int(j0)) % n).astype(np.float64) / n
    dtilde += amplitude * np.asarray(stilde, dtype=np.complex128) * np.exp(-2j * math.pi * ph)
    return dtilde


def sample_masses(seed: int, stream: int, count: int, lo: float, hi: float, log: bool):
    """(m1, m2) in solar masses, iid uniform in [lo, hi] or in [ln lo, ln hi]."""
    u = uniform(seed, stream, 2 * count)
    if log:
        m = np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    else:
        m = lo + u * (hi - lo)
    return m[:count].copy(), m[count:].copy()


def injection_times(seed: int, stream: int, count: int, lo: int, hi: int, min_sep: int):
    """``count`` integer sample indices in [lo, hi), pairwise at least
    ``min_sep`` apart (circular distance), drawn by rejection in order."""
    out: list[int] = []
    span = hi - lo
    i = 0
    while len(out) < count:
        if i > 10000 * (count + 1):
            raise ValueError("cannot place injections with that separation")
        u = float(uniform(seed, stream, 1, i)[0])
        i += 1
        j = lo + min(int(u * span), span - 1)
        if all(min(abs(j - o), span - abs(j - o)) >= min_sep for o in out):
            out.append(j)
    return np.asarray(out, dtype=np.int64)


def injection_snrs(seed: int, stream: int, count: int, lo: float, hi: float):
    return lo + uniform(seed, stream, count) * (hi - lo)


@dataclass(frozen=True)
class Workload:
    """A synthetic workload: segment shape, template bank recipe, injections."""

    name: str
    n: int
    fs: float
    f_low: float
    pn_x2: int
    n_templates: int
    mass_lo: float
    mass_hi: float
    mass_log: bool
    n_inj: int
    snr_lo: float
    snr_hi: float
    psd_scale: float
    seed: int

    @property
    def df(self) -> float:
        return self.fs / self.n

    def psd(self):
        return psd_onesided(self.n, self.fs, self.psd_scale)

    def masses(self):
        return sample_masses(self.seed, 1, self.n_templates, self.mass_lo, self.mass_hi, self.mass_log)

    def noise(self, segment: int = 0):
        return noise_spectrum(self.seed, 1000 + segment, self.n, self.fs, self.psd(), self.f_low)

    def injection_plan(self, segment: int = 0):
        """(template indices, sample offsets j0, target SNRs) of the injections,
        each an exact member of the bank."""
        if self.n_inj == 0:
            z = np.zeros(0, dtype=np.int64)
            return z, z, np.zeros(0)
        u = uniform(self.seed, 2000 + segment, self.n_inj)
        tmpl = np.minimum((u * self.n_templates).astype(np.int64), self.n_templates - 1)
        sep = int(2 * self.fs)
        j0 = injection_times(self.seed, 3000 + segment, self.n_inj, 0, self.n, sep)
        snr = injection_snrs(self.seed, 4000 + segment, self.n_inj, self.snr_lo, self.snr_hi)
        return tmpl, j0, snr


def _w(name, n, f_low, pn_x2, nt, lo, hi, log, ninj, slo, shi, psd_scale, c):
    return Workload(name, n, 4096.0, f_low, pn_x2, nt, lo, hi, log, ninj, slo, shi,
                    psd_scale, 1006_4644 + c)


# Workload recipes (sizes and ranges of the five stated workloads).
WORKLOADS = {
    "seg16s_bank64_pn2": _w("seg16s_bank64_pn2", 1 << 16, 40.0, 4, 64, 1.0, 3.0, False, 1, 12.0, 12.0, 1.0, 1),
    "seg256s_bank1024_pn35": _w("seg256s_bank1024_pn35", 1 << 20, 30.0, 7, 1024, 1.0, 10.0, False, 5, 8.0, 15.0, 1.0, 2),
    "seg256s_bank10k_pn35": _w("seg256s_bank10k_pn35", 1 << 20, 20.0, 7, 10000, 1.0, 25.0, True, 5, 8.0, 15.0, 1.0, 3),
    "seg1024s_bank10k_pn35": _w("seg1024s_bank10k_pn35", 1 << 22, 20.0, 7, 10000, 1.0, 25.0, True, 5, 8.0, 15.0, 1.0, 3),
    "seg1024s_bank1m_et": _w("seg1024s_bank1m_et", 1 << 22, 10.0, 7, 1_000_000, 1.0, 50.0, True, 5, 8.0, 15.0, 1e-4, 5),
}
