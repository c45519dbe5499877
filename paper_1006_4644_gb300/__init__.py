"""GB300 bank matched filter for coalescing-binary searches.

A thin Python layer over the C ABI in ``include/cui.h`` (``libcui.so``).  The
CUDA library does all of the work: segment transform, template generation,
correlation, inverse FFT, peak and trigger reduction.  This module only
marshals arguments; PyTorch, when used, supplies device memory and streams.

    bank = Bank(m1, m2, n=1 << 20, fs=4096.0, f_low=30.0, pn_x2=7)
    bank.upload(strain, psd)          # numpy (host) or torch float64 (device)
    bank.filter()
    peaks = bank.peaks()               # structured array: sample, snr, phase
    trig, total = bank.triggers()
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (CUI_PLAIN, CUI_PLAIN_FP64, CUI_PSI_FP64, CUI_STORE_BF16, PEAK_DTYPE, TRIGGER_DTYPE, CuiError,
                   cui_bank_desc)

__all__ = ["Bank", "Prescreen", "Regions", "prescreen_rank", "ensemble_scores", "template_bands", "CuiError", "CUI_PSI_FP64", "CUI_STORE_BF16", "CUI_PLAIN",
           "CUI_PLAIN_FP64", "PEAK_DTYPE", "TRIGGER_DTYPE", "load"]

load = _lib.load


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


class Bank:
    """One template bank on the current CUDA device (cui_bank_create)."""

    def __init__(self, m1, m2, *, n: int, fs: float, f_low: float, pn_x2: int, flags: int = 0,
                 snr_threshold: float = 6.0, window: int | None = None, valid: tuple[int, int | None] = (0, None),
                 trigger_capacity: int = 0, stream=None):
        self._l = _lib.load()
        m1 = np.ascontiguousarray(m1, dtype=np.float64)
        m2 = np.ascontiguousarray(m2, dtype=np.float64)
        if m1.shape != m2.shape or m1.ndim != 1:
            raise ValueError("m1 and m2 must be 1-D arrays of equal length")
        self.n, self.fs, self.n_templates = int(n), float(fs), len(m1)
        self.stream = _current_stream() if stream is None else int(stream)
        d = cui_bank_desc()
        d.pn_order_x2, d.f_low, d.sample_rate, d.n, d.flags = int(pn_x2), float(f_low), float(fs), int(n), int(flags)
        d.snr_threshold = float(snr_threshold)
        d.window = int(fs) if window is None else int(window)
        d.valid_lo = int(valid[0])
        d.valid_hi = int(n) if valid[1] is None else int(valid[1])
        d.trigger_capacity = int(trigger_capacity)
        d.stream = self.stream
        self.desc = d
        h = C.c_void_p()
        _lib.check(self._l.cui_bank_create(C.byref(d), m1.ctypes.data, m2.ctypes.data, len(m1), C.byref(h)),
                   "cui_bank_create")
        self._h = h

    # -- segment -------------------------------------------------------------
    def upload(self, strain, psd):
        """strain: N float64 samples; psd: N/2+1 float64 values (1/Hz).  Both
        host numpy arrays, or both device torch tensors."""
        if _is_torch(strain):
            if not (strain.is_cuda and psd.is_cuda):
                # host tensors go through numpy
                return self.upload(strain.numpy(), psd.numpy())
            if not (strain.is_contiguous() and psd.is_contiguous()):
                raise ValueError("device tensors must be contiguous")
            self._keep = (strain, psd)
            st = self._l.cui_segment_upload(self._h, strain.data_ptr(), strain.numel(), psd.data_ptr(),
                                            psd.numel(), 1)
        else:
            strain = np.ascontiguousarray(strain, dtype=np.float64)
            psd = np.ascontiguousarray(psd, dtype=np.float64)
            self._keep = (strain, psd)
            st = self._l.cui_segment_upload(self._h, strain.ctypes.data, strain.size, psd.ctypes.data, psd.size, 0)
        _lib.check(st, "cui_segment_upload")

    # -- filtering -----------------------------------------------------------
    def filter(self, order=None, peaks_dev=None):
        """Filter the bank (or ``order``, template indices) against the
        uploaded segment.  ``peaks_dev``: optional device tensor of at least
        16 * n_templates bytes receiving the peaks."""
        if order is None:
            optr, cnt = None, self.n_templates
        else:
            self._order = np.ascontiguousarray(order, dtype=np.int32)
            optr, cnt = self._order.ctypes.data, self._order.size
        pptr = None if peaks_dev is None else peaks_dev.data_ptr()
        _lib.check(self._l.cui_filter_bank(self._h, optr, cnt, pptr), "cui_filter_bank")

    def peaks(self, count: int | None = None):
        count = self.n_templates if count is None else int(count)
        out = np.zeros(count, dtype=PEAK_DTYPE)
        _lib.check(self._l.cui_peaks(self._h, out.ctypes.data, count), "cui_peaks")
        return out

    def triggers(self, capacity: int = 1 << 20, allow_overflow: bool = False):
        """(triggers sorted by (tmpl, sample), exact total)."""
        buf = getattr(self, "_trig_buf", None)
        if buf is None or len(buf) < capacity:
            buf = self._trig_buf = np.empty(capacity, dtype=TRIGGER_DTYPE)  # reused across calls
        out = buf[:capacity]
        tot = C.c_int64()
        st = self._l.cui_triggers(self._h, out.ctypes.data, capacity, C.byref(tot))
        if not (allow_overflow and st == _lib.CUI_ERR_OVERFLOW):
            _lib.check(st, "cui_triggers")
        dev_cap = self.desc.trigger_capacity or (1 << 20)
        return out[: min(tot.value, capacity, dev_cap)].copy(), tot.value

    def results(self, capacity: int = 1 << 20, allow_overflow: bool = False):
        """(peaks, triggers, exact trigger total) of the last filter call, read
        back together (cui_results: one synchronisation in the common case)."""
        peaks = np.zeros(self.n_templates, dtype=PEAK_DTYPE)
        buf = getattr(self, "_trig_buf", None)
        if buf is None or len(buf) < capacity:
            buf = self._trig_buf = np.empty(capacity, dtype=TRIGGER_DTYPE)
        out = buf[:capacity]
        tot = C.c_int64()
        st = self._l.cui_results(self._h, peaks.ctypes.data, self.n_templates, out.ctypes.data, capacity,
                                 C.byref(tot))
        if not (allow_overflow and st == _lib.CUI_ERR_OVERFLOW):
            _lib.check(st, "cui_results")
        dev_cap = self.desc.trigger_capacity or (1 << 20)
        return peaks, out[: min(tot.value, capacity, dev_cap)].copy(), tot.value

    def clustered_triggers(self, capacity: int = 1 << 20):
        """Loudest trigger of each window over the whole bank (last filter call),
        in increasing sample order; ties go to the lower sample, then template."""
        out = np.empty(capacity, dtype=TRIGGER_DTYPE)
        tot = C.c_int64()
        _lib.check(self._l.cui_cluster_triggers(self._h, out.ctypes.data, capacity, C.byref(tot)),
                   "cui_cluster_triggers")
        return out[: tot.value].copy()

    def trigger_chisq(self, trig, bands: int = 16):
        """(chi^2, rho) at trigger records (structured array as returned by
        ``triggers``): the equal-power sub-band signal-consistency test."""
        trig = np.ascontiguousarray(trig, dtype=TRIGGER_DTYPE)
        chi = np.zeros(len(trig), dtype=np.float32)
        rho = np.zeros(len(trig), dtype=np.float32)
        _lib.check(self._l.cui_trigger_chisq(self._h, int(bands), trig.ctypes.data, len(trig), chi.ctypes.data,
                                             rho.ctypes.data), "cui_trigger_chisq")
        return chi, rho

    def set_band(self, f_lo: float = 0.0, f_hi: float = 0.0):
        """Restrict later filter calls to each template's bins in [f_lo, f_hi)
        (f_hi <= 0: no upper limit; set_band() restores the full band)."""
        _lib.check(self._l.cui_bank_set_band(self._h, float(f_lo), float(f_hi)), "cui_bank_set_band")

    def band_correlate(self, tmpl, t_sec, f_lo: float = 0.0, f_hi: float = 0.0):
        """(z, sigma^2) of templates tmpl[i] at times t_sec[i] (seconds after the
        segment's first sample) over the band [f_lo, f_hi), by direct sums, in
        physical units: complex128 z and float64 sigma^2 arrays."""
        tm = np.ascontiguousarray(tmpl, dtype=np.int32)
        ts = np.ascontiguousarray(t_sec, dtype=np.float64)
        if tm.shape != ts.shape:
            raise ValueError("tmpl and t_sec must have the same length")
        z = np.zeros(2 * len(tm))
        s2 = np.zeros(len(tm))
        _lib.check(self._l.cui_band_correlate(self._h, tm.ctypes.data, ts.ctypes.data, len(tm), float(f_lo),
                                              float(f_hi), z.ctypes.data, s2.ctypes.data), "cui_band_correlate")
        return z[0::2] + 1j * z[1::2], s2

    def band_combine(self, t_high, low: "Bank", t_low, tmpl, f_split: float):
        """Candidates detected by this bank (band [f_split, ...)) at t_high[i]
        completed by `low` over [..., f_split) at t_low[i] and added coherently
        (cui_band_combine): (rho, phase, sums [n, 6] = Re z_h, Im z_h,
        sigma_h^2, Re z_l, Im z_l, sigma_l^2)."""
        tm = np.ascontiguousarray(tmpl, dtype=np.int32)
        th = np.ascontiguousarray(t_high, dtype=np.float64)
        tl = np.ascontiguousarray(t_low, dtype=np.float64)
        if not (tm.shape == th.shape == tl.shape):
            raise ValueError("tmpl, t_high and t_low must have the same length")
        rho, ph, sums = np.zeros(len(tm)), np.zeros(len(tm)), np.zeros((len(tm), 6))
        _lib.check(self._l.cui_band_combine(self._h, th.ctypes.data, low._h, tl.ctypes.data, tm.ctypes.data, len(tm),
                                            float(f_split), rho.ctypes.data, ph.ctypes.data, sums.ctypes.data),
                   "cui_band_combine")
        return rho, ph, sums

    def band_series(self, out_dev, f_lo: float = 0.0, f_hi: float = 0.0, decim: int = 1):
        """Write the uploaded segment restricted to [f_lo, f_hi) at the sample
        rate fs / decim into a float64 device tensor of N / decim samples."""
        if out_dev.numel() != self.n // max(1, int(decim)) or str(out_dev.dtype) != "torch.float64" \
                or not out_dev.is_contiguous():
            raise ValueError("out_dev must be a contiguous float64 device tensor of N / decim samples")
        _lib.check(self._l.cui_segment_band_series(self._h, float(f_lo), float(f_hi), int(decim), out_dev.data_ptr()),
                   "cui_segment_band_series")

    def td_template(self, t: int, hp_dev, hx_dev, pn_x2: int = 5):
        """Write the time-domain polarisations of template t (the paper's
        generator form, TaylorT2, up to 2.5PN) into float64 device tensors of
        N samples."""
        _lib.check(self._l.cui_td_template(self._h, int(t), int(pn_x2), hp_dev.data_ptr(), hx_dev.data_ptr()),
                   "cui_td_template")

    def sigma(self):
        out = np.zeros(self.n_templates)
        _lib.check(self._l.cui_bank_sigma(self._h, out.ctypes.data), "cui_bank_sigma")
        return out

    def template(self, t: int, out_dev):
        """Write h~_k (k = 0..N/2) of template t into a complex64 device tensor."""
        _lib.check(self._l.cui_bank_template(self._h, int(t), out_dev.data_ptr()), "cui_bank_template")

    # -- tiling ----------------------------------------------------------------
    def tuning(self) -> dict:
        tu = _lib.cui_tuning()
        _lib.check(self._l.cui_bank_get_tuning(self._h, C.byref(tu)), "cui_bank_get_tuning")
        return tu.as_dict()

    def set_tuning(self, n1: int, ccols: int, rpc: int, batch: int):
        tu = _lib.cui_tuning(int(n1), int(ccols), int(rpc), int(batch))
        _lib.check(self._l.cui_bank_set_tuning(self._h, C.byref(tu)), "cui_bank_set_tuning")

    def set_wait_bounds(self, cas_rounds: int = -1, copy_wait_ns: int = -1):
        """Lower the bounds of the device waits (for tests of the error path);
        negative values restore the defaults."""
        _lib.check(self._l.cui_bank_set_wait_bounds(self._h, int(cas_rounds), int(copy_wait_ns)),
                   "cui_bank_set_wait_bounds")

    def autotune(self, reps: int = 2):
        """Time every tiling with kernels at this N on the uploaded segment,
        keep the fastest; returns (tiling, ms per filter call)."""
        tu, ms = _lib.cui_tuning(), C.c_double()
        _lib.check(self._l.cui_bank_autotune(self._h, int(reps), C.byref(tu), C.byref(ms)), "cui_bank_autotune")
        return tu.as_dict(), ms.value

    def trace(self, level: int = 1):
        """Record CUDA events around the kernel groups of later calls: level 1
        per call group (the fused filter stays one graph launch), level 2 per
        fused kernel group (direct launches), 0 off."""
        _lib.check(self._l.cui_trace_enable(self._h, int(level)), "cui_trace_enable")

    def trace_read(self) -> dict:
        """{group: (kernel launches, timed intervals, total ms)} since the last read."""
        buf = (_lib.cui_trace_stat * 8)()
        n = C.c_int64()
        _lib.check(self._l.cui_trace_read(self._h, buf, 8, C.byref(n)), "cui_trace_read")
        return {buf[i].name.decode(): (buf[i].launches, buf[i].calls, buf[i].ms) for i in range(n.value)}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._l.cui_bank_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def prescreen_rank(m1, m2, scores, top_k: int | None = None):
    """Template order for ``Bank.filter``: the chirp-mass regions of the bank
    (as many as ``scores`` has entries) by descending score, the first
    ``top_k`` of them (all by default) (cui_prescreen_rank)."""
    m1 = np.ascontiguousarray(m1, dtype=np.float64)
    m2 = np.ascontiguousarray(m2, dtype=np.float64)
    sc = np.ascontiguousarray(scores, dtype=np.float32).reshape(-1)
    if m1.shape != m2.shape or m1.ndim != 1:
        raise ValueError("m1 and m2 must be 1-D arrays of one length")
    regions = len(sc)
    k = regions if top_k is None else int(top_k)
    out = np.empty(max(len(m1), 1), dtype=np.int32)
    cnt = C.c_int64()
    lib = _lib.load_prescreen(_lib.load())
    _lib.check(lib.cui_prescreen_rank(m1.ctypes.data, m2.ctypes.data, len(m1), sc.ctypes.data, regions, k,
                                      out.ctypes.data, C.byref(cnt)), "cui_prescreen_rank")
    return out[: cnt.value].copy()


class Regions:
    """A bank's region plan (cui_regions_*): the bank sorted by chirp mass and
    cut into equal-count regions once; order(scores, top_k) is then the
    template order of the top_k best-scored regions, as prescreen_rank gives."""

    def __init__(self, m1, m2, regions: int = 100):
        self._l = _lib.load_prescreen(_lib.load())
        a1 = np.ascontiguousarray(m1, dtype=np.float64)
        a2 = np.ascontiguousarray(m2, dtype=np.float64)
        if a1.shape != a2.shape:
            raise ValueError("m1 and m2 must have the same length")
        h = C.c_void_p()
        _lib.check(self._l.cui_regions_create(a1.ctypes.data, a2.ctypes.data, len(a1), int(regions), C.byref(h)),
                   "cui_regions_create")
        self._h, self.regions, self.n_templates = h, int(regions), len(a1)
        self._out = np.empty(len(a1), dtype=np.int32)

    def order(self, scores, top_k: int | None = None):
        sc = np.ascontiguousarray(scores, dtype=np.float32)
        if sc.shape != (self.regions,):
            raise ValueError("one score per region")
        cnt = C.c_int64()
        k = self.regions if top_k is None else int(top_k)
        _lib.check(self._l.cui_regions_order(self._h, sc.ctypes.data, k, self._out.ctypes.data, C.byref(cnt)),
                   "cui_regions_order")
        return self._out[:cnt.value].copy()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._l.cui_regions_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def template_bands(m1, m2, *, n: int, fs: float, f_low: float):
    """(k_low, k_hi per template) by the library's rule (cui_template_bands;
    host only, no GPU)."""
    lib = _lib.load()
    a1 = np.ascontiguousarray(m1, dtype=np.float64)
    a2 = np.ascontiguousarray(m2, dtype=np.float64)
    if a1.shape != a2.shape:
        raise ValueError("m1 and m2 must have the same length")
    khi = np.zeros(len(a1), dtype=np.int32)
    klo = C.c_int32()
    _lib.check(lib.cui_template_bands(a1.ctypes.data, a2.ctypes.data, len(a1), int(n), float(fs), float(f_low),
                                      C.byref(klo), khi.ctypes.data), "cui_template_bands")
    return int(klo.value), khi


def ensemble_scores(nets, feat_dev, out_dev):
    """Mean over the networks of their region probabilities (softmax of the
    scores) for feature rows [count, bands, frames] into out_dev [count,
    regions] (cui_prescreen_ensemble_scores)."""
    if not nets:
        raise ValueError("no networks")
    lib = nets[0]._l
    arr = (C.c_void_p * len(nets))(*[p._h.value for p in nets])
    _lib.check(lib.cui_prescreen_ensemble_scores(arr, len(nets), feat_dev.data_ptr(), feat_dev.shape[0],
                                                 out_dev.data_ptr()), "cui_prescreen_ensemble_scores")


class Prescreen:
    """The learned region prescreen (cui_prescreen_*): whitened band-power
    features, a conv1d + MLP scorer, and its training on the GPU.  Device
    arrays are torch tensors (float32 features [count, bands, frames], targets
    and scores [count, regions]; complex128 data spectra [count, n/2 + 1])."""

    def __init__(self, *, n: int, fs: float, f_low: float, bands: int = 16, frame: int | None = None, regions: int = 100,
                 max_batch: int = 256, lr: float = 1e-3, betas=(0.9, 0.999), eps: float = 1e-8, seed: int = 1,
                 stream=None):
        self._l = _lib.load_prescreen(_lib.load())
        d = _lib.cui_prescreen_desc()
        frame = max(1, int(n) // 256) if frame is None else frame  # the finest frames the network takes
        d.n, d.sample_rate, d.f_low, d.bands, d.frame, d.regions = int(n), float(fs), float(f_low), bands, frame, regions
        d.max_batch, d.lr, d.beta1, d.beta2, d.eps, d.seed = max_batch, lr, betas[0], betas[1], eps, int(seed)
        d.stream = _current_stream() if stream is None else int(stream)
        self.desc = d
        h = C.c_void_p()
        _lib.check(self._l.cui_prescreen_create(C.byref(d), C.byref(h)), "cui_prescreen_create")
        self._h = h
        npar, frames = C.c_int64(), C.c_int32()
        _lib.check(self._l.cui_prescreen_info(h, C.byref(npar), C.byref(frames)), "cui_prescreen_info")
        self.n_params, self.frames, self.bands, self.regions = npar.value, frames.value, bands, regions

    def features(self, dtilde_dev, psd_dev, out_dev):
        count = dtilde_dev.shape[0] if dtilde_dev.dim() == 2 else 1
        _lib.check(self._l.cui_prescreen_features(self._h, dtilde_dev.data_ptr(), psd_dev.data_ptr(), count,
                                                  out_dev.data_ptr()), "cui_prescreen_features")

    def bank_features(self, bank: "Bank", out_dev):
        _lib.check(self._l.cui_prescreen_bank_features(self._h, bank._h, out_dev.data_ptr()),
                   "cui_prescreen_bank_features")

    def scores(self, feat_dev, out_dev):
        _lib.check(self._l.cui_prescreen_scores(self._h, feat_dev.data_ptr(), feat_dev.shape[0], out_dev.data_ptr()),
                   "cui_prescreen_scores")

    def train_step(self, feat_dev, target_dev, want_loss: bool = True):
        loss = C.c_float()
        _lib.check(self._l.cui_prescreen_train_step(self._h, feat_dev.data_ptr(), target_dev.data_ptr(),
                                                    feat_dev.shape[0], C.byref(loss) if want_loss else None),
                   "cui_prescreen_train_step")
        return loss.value if want_loss else None

    def gradient(self, feat_dev, target_dev, grad_dev):
        loss = C.c_float()
        _lib.check(self._l.cui_prescreen_gradient(self._h, feat_dev.data_ptr(), target_dev.data_ptr(),
                                                  feat_dev.shape[0], grad_dev.data_ptr(), C.byref(loss)),
                   "cui_prescreen_gradient")
        return loss.value

    def get_state(self):
        th, m, v = (np.zeros(self.n_params, dtype=np.float32) for _ in range(3))
        st = C.c_int64()
        _lib.check(self._l.cui_prescreen_get_state(self._h, th.ctypes.data, m.ctypes.data, v.ctypes.data,
                                                   C.byref(st)), "cui_prescreen_get_state")
        return th, m, v, st.value

    def set_state(self, theta, m=None, v=None, step: int = 0):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        mm = None if m is None else np.ascontiguousarray(m, dtype=np.float32)
        vv = None if v is None else np.ascontiguousarray(v, dtype=np.float32)
        _lib.check(self._l.cui_prescreen_set_state(self._h, th.ctypes.data, None if mm is None else mm.ctypes.data,
                                                   None if vv is None else vv.ctypes.data, int(step)),
                   "cui_prescreen_set_state")

    def fit_norm(self, feat_dev):
        """Set the per-band feature standardisation from these feature rows."""
        _lib.check(self._l.cui_prescreen_fit_norm(self._h, feat_dev.data_ptr(), feat_dev.shape[0]),
                   "cui_prescreen_fit_norm")

    def get_norm(self):
        mean, sd = np.zeros(self.bands, dtype=np.float32), np.zeros(self.bands, dtype=np.float32)
        _lib.check(self._l.cui_prescreen_get_norm(self._h, mean.ctypes.data, sd.ctypes.data), "cui_prescreen_get_norm")
        return mean, sd

    def set_norm(self, mean, sd):
        mean = np.ascontiguousarray(mean, dtype=np.float32)
        sd = np.ascontiguousarray(sd, dtype=np.float32)
        _lib.check(self._l.cui_prescreen_set_norm(self._h, mean.ctypes.data, sd.ctypes.data), "cui_prescreen_set_norm")

    def save(self, path: str):
        """Checkpoint: JSON header line, then parameters, Adam moments and the
        feature standardisation (mean, std per band), all FP32."""
        import json

        th, m, v, st = self.get_state()
        mean, sd = self.get_norm()
        hdr = {"n_params": self.n_params, "step": st, "bands": self.bands, "frames": self.frames,
               "regions": self.regions, "n": self.desc.n, "frame": self.desc.frame, "norm": True}
        with open(path, "wb") as fh:
            fh.write((json.dumps(hdr) + "\n").encode())
            fh.write(th.tobytes() + m.tobytes() + v.tobytes() + mean.tobytes() + sd.tobytes())

    def load(self, path: str):
        import json

        with open(path, "rb") as fh:
            hdr = json.loads(fh.readline())
            if hdr["n_params"] != self.n_params or hdr["bands"] != self.bands:
                raise ValueError("checkpoint does not match this network")
            raw = np.frombuffer(fh.read(), dtype=np.float32)
        a = raw[:3 * self.n_params].reshape(3, self.n_params)
        self.set_state(a[0], a[1], a[2], hdr["step"])
        if hdr.get("norm"):
            rest = raw[3 * self.n_params:]
            self.set_norm(rest[:self.bands], rest[self.bands:2 * self.bands])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._l.cui_prescreen_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
