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

__all__ = ["Bank", "CuiError", "CUI_PSI_FP64", "CUI_STORE_BF16", "CUI_PLAIN", "CUI_PLAIN_FP64", "PEAK_DTYPE",
           "TRIGGER_DTYPE", "load"]

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
        out = np.zeros(capacity, dtype=TRIGGER_DTYPE)
        tot = C.c_int64()
        st = self._l.cui_triggers(self._h, out.ctypes.data, capacity, C.byref(tot))
        if not (allow_overflow and st == _lib.CUI_ERR_OVERFLOW):
            _lib.check(st, "cui_triggers")
        dev_cap = self.desc.trigger_capacity or (1 << 20)
        return out[: min(tot.value, capacity, dev_cap)].copy(), tot.value

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

    def autotune(self, reps: int = 2):
        """Time every tiling with kernels at this N on the uploaded segment,
        keep the fastest; returns (tiling, ms per filter call)."""
        tu, ms = _lib.cui_tuning(), C.c_double()
        _lib.check(self._l.cui_bank_autotune(self._h, int(reps), C.byref(tu), C.byref(ms)), "cui_bank_autotune")
        return tu.as_dict(), ms.value

    def trace(self, on: bool = True):
        """Record CUDA events around every kernel group of later calls."""
        _lib.check(self._l.cui_trace_enable(self._h, int(bool(on))), "cui_trace_enable")

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
