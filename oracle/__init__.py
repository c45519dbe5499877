"""FP64 CPU oracle of the bank matched filter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library under ``paper_1006_4644_gb300`` never
imports, links or calls it, and the two share no code.

The arithmetic lives in ``cui_oracle.c`` (plain C, FP64, compiled with gcc on
first use into ``oracle/_build``); this module only marshals numpy arrays.
Each function names the part of the paper it follows:

* ``segment_spectrum``  -- X(f) of eq:matchedfilter, d~_k = dt sum_j d_j e^{-2 pi i jk/N}
* ``spa_phase`` / ``spa_template`` -- the post-Newtonian template of Sec.
  "template generation", in its stationary-phase (TaylorF2) form
* ``sigma2``           -- the normalisation <theta, theta> of step 1 of the
  per-chunk loop (Sec. "Matched filtering")
* ``correlate``        -- eq:matchedfilter on the sampled one-sided band
* ``correlate_polarisations`` -- steps 2-3 of the per-chunk loop (two real
  correlators c_+, c_x)
* ``peak_triggers``    -- step 4 of the per-chunk loop (maximum above a
  threshold), with the window reading of "local maximum"
* ``cluster_windows``  -- the final reduction of the per-template maxima
  across the bank (Sec. "Matched filtering", last step), with the same window
  reading: per window, the loudest trigger over all templates
* ``chisq``            -- the chi-squared signal-consistency test that the
  paper lists as future work (Sec. "Conclusions"), in its equal-power
  sub-band form: chi^2 = p sum_l |z_l - z/p|^2 / sigma^2
* ``band_edges`` / ``band_filter_template`` / ``band_correlate`` /
  ``band_series`` -- the multi-band search of Sec. "Online analysis
  considerations" (the band split, the filter restricted to one band, the band
  correlators summed directly at any time, which add up across bands and
  segments, and the data restricted to a band and resampled)
* ``fft`` / ``dft``    -- textbook radix-2 FFT and naive DFT used above

The absolute constant of Psi (the -pi/4 of the stationary phase and the
constant part of the 2.5PN logarithm, referred to v_lso) is pinned by a direct
Fourier transform of the time-domain chirp of ``oracle.td``: zero offset below
2.5PN, 9 alpha_5 ln 6 / (256 eta) at 2.5PN (tests/test_oracle_phase_constant.py).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cui_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
# A prebuilt oracle library to load instead (the mutation tests point this at
# deliberately broken copies of cui_oracle.c).
_OVERRIDE = os.environ.get("CUI_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_L = C.c_long
_D = C.c_double
_PL = C.POINTER(C.c_long)
_PD = C.POINTER(C.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic) if stale."""
    with _lock:
        stale = force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC)
        if stale:
            os.makedirs(os.path.dirname(_OUT), exist_ok=True)
            tmp = _OUT + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(_OVERRIDE or build())
    lib.or_dft.argtypes = [_L, C.c_int, _dp, _dp, _dp, _dp]
    lib.or_dft.restype = None
    lib.or_fft.argtypes = [_L, C.c_int, _dp, _dp]
    lib.or_fft.restype = C.c_int
    lib.or_segment_spectrum.argtypes = [_L, _D, _dp, _dp, _dp]
    lib.or_segment_spectrum.restype = C.c_int
    lib.or_spa_phase.argtypes = [_D, _D, C.c_int, _L, _dp, _dp]
    lib.or_spa_phase.restype = None
    lib.or_template_band.argtypes = [_D, _D, _D, _D, _L, _PL, _PL]
    lib.or_template_band.restype = None
    lib.or_spa_template.argtypes = [_D, _D, C.c_int, _D, _D, _L, _dp, _dp, _PL, _PL]
    lib.or_spa_template.restype = C.c_int
    lib.or_sigma2.argtypes = [_L, _D, _dp, _dp, _dp, _L, _L]
    lib.or_sigma2.restype = _D
    lib.or_correlate.argtypes = [_L, _D, _dp, _dp, _dp, _dp, _dp, _L, _L, _dp, _dp]
    lib.or_correlate.restype = C.c_int
    lib.or_correlate_polarisations.argtypes = [_L, _D, _dp, _dp, _dp, _dp, _dp, _L, _L, _dp, _dp]
    lib.or_correlate_polarisations.restype = C.c_int
    lib.or_peak_triggers.argtypes = [_L, _dp, _dp, _D, _L, _L, _L, _D, _PL, _PD, _PD, _lp, _dp, _dp, _L]
    lib.or_peak_triggers.restype = _L
    lib.or_filter_template.argtypes = [_L, _D, _dp, _dp, _dp, _D, _D, C.c_int, _D, _L, _L, _L, _D,
                                       _PD, _PL, _PD, _PD, _lp, _dp, _dp, _L]
    lib.or_filter_template.restype = _L
    _lib = lib
    return lib


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _split(z):
    z = np.asarray(z, dtype=np.complex128)
    return _f64(z.real), _f64(z.imag)


def dft(x, sign: int):
    """Naive O(n^2) DFT, y_k = sum_j x_j exp(sign 2 pi i jk/n)."""
    xr, xi = _split(x)
    n = len(xr)
    yr, yi = np.empty(n), np.empty(n)
    _load().or_dft(n, int(sign), xr, xi, yr, yi)
    return yr + 1j * yi


def fft(x, sign: int):
    """Radix-2 FFT with the same convention as ``dft`` (n a power of two)."""
    xr, xi = _split(x)
    xr, xi = xr.copy(), xi.copy()
    if _load().or_fft(len(xr), int(sign), xr, xi) != 0:
        raise ValueError("n must be a power of two")
    return xr + 1j * xi


def segment_spectrum(d, fs: float):
    """d~_k = dt sum_j d_j exp(-2 pi i jk/n) for k = 0..n/2."""
    d = _f64(d)
    n = len(d)
    dr, di = np.empty(n // 2 + 1), np.empty(n // 2 + 1)
    if _load().or_segment_spectrum(n, float(fs), d, dr, di) != 0:
        raise ValueError("n must be a power of two")
    return dr + 1j * di


def spa_phase(m1: float, m2: float, pn_x2: int, f):
    f = _f64(np.atleast_1d(f))
    out = np.empty_like(f)
    _load().or_spa_phase(float(m1), float(m2), int(pn_x2), len(f), f, out)
    return out


def template_band(m1: float, m2: float, f_low: float, fs: float, n: int):
    lo, hi = C.c_long(), C.c_long()
    _load().or_template_band(float(m1), float(m2), float(f_low), float(fs), int(n), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def spa_template(m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int):
    """(h~_k for k = 0..n/2, k_lo, k_hi)."""
    hr, hi = np.empty(n // 2 + 1), np.empty(n // 2 + 1)
    lo, kh = C.c_long(), C.c_long()
    if _load().or_spa_template(float(m1), float(m2), int(pn_x2), float(f_low), float(fs), int(n),
                               hr, hi, C.byref(lo), C.byref(kh)) != 0:
        raise MemoryError("oracle template")
    return hr + 1j * hi, lo.value, kh.value


def sigma2(h, psd, fs: float, n: int, k_lo: int, k_hi: int) -> float:
    hr, hi = _split(h)
    return float(_load().or_sigma2(int(n), float(fs), hr, hi, _f64(psd), int(k_lo), int(k_hi)))


def correlate(dtilde, h, psd, fs: float, n: int, k_lo: int, k_hi: int):
    """z_j, j = 0..n-1 (complex128)."""
    dr, di = _split(dtilde)
    hr, hi = _split(h)
    zr, zi = np.empty(n), np.empty(n)
    if _load().or_correlate(int(n), float(fs), dr, di, hr, hi, _f64(psd), int(k_lo), int(k_hi), zr, zi) != 0:
        raise ValueError("n must be a power of two")
    return zr + 1j * zi


def correlate_polarisations(dtilde, h, psd, fs: float, n: int, k_lo: int, k_hi: int):
    """(c_plus, c_cross), the paper's two real correlators."""
    dr, di = _split(dtilde)
    hr, hi = _split(h)
    cp, cx = np.empty(n), np.empty(n)
    if _load().or_correlate_polarisations(int(n), float(fs), dr, di, hr, hi, _f64(psd), int(k_lo),
                                          int(k_hi), cp, cx) != 0:
        raise ValueError("n must be a power of two")
    return cp, cx


def peak_triggers(z, sig2: float, lo: int, hi: int, window: int, thr: float, cap: int = 1 << 16):
    zr, zi = _split(z)
    pj, pr, pp = C.c_long(), C.c_double(), C.c_double()
    tj, tr, tp = np.empty(cap, dtype=np.int64), np.empty(cap), np.empty(cap)
    cnt = _load().or_peak_triggers(len(zr), zr, zi, float(sig2), int(lo), int(hi), int(window), float(thr),
                                   C.byref(pj), C.byref(pr), C.byref(pp), tj, tr, tp, int(cap))
    m = min(cnt, cap)
    return dict(peak_j=pj.value, peak_rho=pr.value, peak_phase=pp.value, n_trig=int(cnt),
                trig_j=tj[:m].copy(), trig_rho=tr[:m].copy(), trig_phase=tp[:m].copy())


def filter_template(dtilde, psd, m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int,
                    lo: int = 0, hi: int | None = None, window: int | None = None, thr: float = 6.0,
                    cap: int = 1 << 16):
    """One template through the per-chunk loop; returns a dict with sigma2,
    the peak (j, rho, phase) and the triggers."""
    hi = n if hi is None else hi
    window = int(fs) if window is None else window
    dr, di = _split(dtilde)
    psd = _f64(psd)
    s2, pj, pr, pp = C.c_double(), C.c_long(), C.c_double(), C.c_double()
    tj, tr, tp = np.empty(cap, dtype=np.int64), np.empty(cap), np.empty(cap)
    cnt = _load().or_filter_template(int(n), float(fs), dr, di, psd, float(m1), float(m2), int(pn_x2),
                                     float(f_low), int(lo), int(hi), int(window), float(thr),
                                     C.byref(s2), C.byref(pj), C.byref(pr), C.byref(pp), tj, tr, tp, int(cap))
    if cnt < 0:
        raise MemoryError("oracle filter")
    m = min(cnt, cap)
    return dict(sigma2=s2.value, peak_j=pj.value, peak_rho=pr.value, peak_phase=pp.value, n_trig=int(cnt),
                trig_j=tj[:m].copy(), trig_rho=tr[:m].copy(), trig_phase=tp[:m].copy())


def filter_bank(dtilde, psd, m1s, m2s, pn_x2: int, f_low: float, fs: float, n: int, lo: int = 0,
                hi: int | None = None, window: int | None = None, thr: float = 6.0, threads: int | None = None):
    """``filter_template`` over a bank, one template per worker thread (the C
    call releases the GIL).  Returns a list of per-template dicts."""
    threads = threads or len(os.sched_getaffinity(0))
    dtilde = np.asarray(dtilde, dtype=np.complex128)
    psd = _f64(psd)
    _load()

    def one(i):
        return filter_template(dtilde, psd, m1s[i], m2s[i], pn_x2, f_low, fs, n, lo, hi, window, thr)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(one, range(len(m1s))))


def cluster_windows(tmpl, sample, rho, lo: int, window: int):
    """Cross-template clustering of trigger records: the windows
    [lo + m W, lo + (m+1) W) are those of the per-template triggers; each
    window keeps its record of largest rho, among equal rho the lowest sample,
    then the lowest template.  Returns the kept record indices in increasing
    sample order.  Plain loops; the records are few."""
    best = {}
    for i in range(len(tmpl)):
        m = (int(sample[i]) - lo) // window
        cand = (float(rho[i]), -int(sample[i]), -int(tmpl[i]))
        if m not in best or cand > best[m][0]:
            best[m] = (cand, i)
    return [best[m][1] for m in sorted(best)]


def chisq(dtilde, psd, m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int, samples, bands: int):
    """chi^2 and rho of one template at the given samples.  The band
    [k_lo, k_hi) is split at k_l = min{k : Pw(k) >= (l/p) Pw(k_hi)}, Pw(k) =
    sum_{k_lo <= j < k} |h~_j|^2 / S_j; z_l(s) = 4 df sum_{k in band l}
    d~_k conj(h~_k) / S_k exp(2 pi i k s / N) by direct summation; z = sum_l z_l;
    chi^2 = p sum_l |z_l - z/p|^2 / sigma^2 and rho = |z| / sigma."""
    h, k_lo, k_hi = spa_template(m1, m2, pn_x2, f_low, fs, n)
    psd = _f64(psd)
    df = fs / n
    k = np.arange(k_lo, k_hi)
    terms = 4.0 * df * np.asarray(dtilde)[k_lo:k_hi] * np.conj(h[k_lo:k_hi]) / psd[k_lo:k_hi]
    power = np.abs(h[k_lo:k_hi]) ** 2 / psd[k_lo:k_hi]
    pw = np.concatenate([[0.0], np.cumsum(power)])  # pw[i] = Pw(k_lo + i)
    edges = [0] + [int(np.searchsorted(pw, pw[-1] * l / bands, side="left")) for l in range(1, bands)] + [len(k)]
    s2 = sigma2(h, psd, fs, n, k_lo, k_hi)
    chi, rho = [], []
    for s in samples:
        ph = np.exp(2j * np.pi * ((k * int(s)) % n) / n)
        zl = np.array([np.sum(terms[edges[l]:edges[l + 1]] * ph[edges[l]:edges[l + 1]]) for l in range(bands)])
        z = zl.sum()
        chi.append(bands * np.sum(np.abs(zl - z / bands) ** 2) / s2)
        rho.append(abs(z) / np.sqrt(s2))
    return np.array(chi), np.array(rho)


def band_edges(m1: float, m2: float, f_low: float, fs: float, n: int, f_lo: float, f_hi: float):
    """[k_a, k_b) of a template cut to the band [f_lo, f_hi): the template's own
    band [k_lo, k_hi) intersected with ceil(f_lo/df) <= k < ceil(f_hi/df)
    (f_hi <= 0: no upper limit); an empty band has k_a == k_b."""
    k_lo, k_hi = template_band(m1, m2, f_low, fs, n)
    df = fs / n
    ka = max(k_lo, int(np.ceil(f_lo / df)))
    kb = k_hi if f_hi <= 0 else min(k_hi, int(np.ceil(f_hi / df)))
    return ka, max(ka, kb)


def band_filter_template(dtilde, psd, m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int,
                         f_lo: float, f_hi: float, lo: int = 0, hi: int | None = None, window: int | None = None,
                         thr: float = 6.0, cap: int = 1 << 16):
    """The per-chunk loop of one template with the template restricted to the
    band [f_lo, f_hi): z_j by the FFT route over the band's bins only, sigma^2
    over the same bins, then the peak and the triggers of rho = |z| / sigma."""
    hi = n if hi is None else hi
    window = int(fs) if window is None else window
    h, _, _ = spa_template(m1, m2, pn_x2, f_low, fs, n)
    ka, kb = band_edges(m1, m2, f_low, fs, n, f_lo, f_hi)
    s2 = sigma2(h, psd, fs, n, ka, kb)
    z = correlate(dtilde, h, psd, fs, n, ka, kb)
    out = peak_triggers(z, s2 if s2 > 0 else 1.0, lo, hi, window, thr, cap)
    out["sigma2"] = s2
    return out


def band_correlate(dtilde, psd, m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int, times,
                   f_lo: float, f_hi: float):
    """(z, sigma^2) of one template over the band [f_lo, f_hi) at arbitrary
    times t (seconds after the segment's first sample), by direct summation:
    z(t) = 4 df sum_{k in band} d~_k conj(h~_k) / S_k exp(2 pi i k df t) and
    sigma^2 = 4 df sum |h~_k|^2 / S_k, in physical units."""
    h, _, _ = spa_template(m1, m2, pn_x2, f_low, fs, n)
    ka, kb = band_edges(m1, m2, f_low, fs, n, f_lo, f_hi)
    psd = _f64(psd)
    df = fs / n
    k = np.arange(ka, kb)
    terms = 4.0 * df * np.asarray(dtilde)[ka:kb] * np.conj(h[ka:kb]) / psd[ka:kb]
    s2 = float(4.0 * df * np.sum(np.abs(h[ka:kb]) ** 2 / psd[ka:kb]))
    z = np.empty(len(times), dtype=np.complex128)
    for i, t in enumerate(times):
        x = (float(t) * df) % 1.0  # t / T mod 1
        z[i] = np.sum(terms * np.exp(2j * np.pi * ((k * x) % 1.0)))
    return z, s2


def band_series(strain, fs: float, f_lo: float, f_hi: float, decim: int):
    """The segment restricted to the bins ceil(f_lo/df) <= k < ceil(f_hi/df)
    below m/2 (f_hi <= 0: up to m/2) at the sample rate fs/decim, m = n/decim:
    x'_j = (1/n) sum_{k in band} X_k e^{2 pi i k j / m} + c.c., X the DFT."""
    n = len(strain)
    m = n // decim
    df = fs / n
    X = segment_spectrum(strain, fs) * fs  # sum_j d_j e^{-2 pi i jk/n}
    k = np.arange(m // 2 + 1)
    ka = max(0, int(np.ceil(f_lo / df)))
    kb = m // 2 if f_hi <= 0 else min(m // 2, int(np.ceil(f_hi / df)))
    Y = np.where((k >= ka) & (k < kb), X[: m // 2 + 1], 0.0)
    return np.fft.irfft(Y, m) * (m / n)
