"""ctypes binding of ``libcui.so`` (include/cui.h).  Argument marshalling only:
every step of the filter runs in the CUDA library.  Loading fails loudly when
the library has not been built; there is no fallback."""

from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcui.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "cui.h")

CUI_OK, CUI_ERR_ARG, CUI_ERR_CUDA, CUI_ERR_OOM, CUI_ERR_STATE, CUI_ERR_OVERFLOW, CUI_ERR_TIMEOUT = range(7)
STATUS_NAMES = {0: "CUI_OK", 1: "CUI_ERR_ARG", 2: "CUI_ERR_CUDA", 3: "CUI_ERR_OOM", 4: "CUI_ERR_STATE",
                5: "CUI_ERR_OVERFLOW", 6: "CUI_ERR_TIMEOUT"}
CUI_PSI_FP64, CUI_STORE_BF16, CUI_PLAIN, CUI_PLAIN_FP64, CUI_NO_GRAPH = 0x1, 0x2, 0x4, 0x8, 0x10


class cui_bank_desc(C.Structure):
    _fields_ = [("pn_order_x2", C.c_int32), ("reserved0", C.c_int32), ("f_low", C.c_double),
                ("sample_rate", C.c_double), ("n", C.c_int64), ("flags", C.c_uint32), ("reserved1", C.c_uint32),
                ("snr_threshold", C.c_double), ("window", C.c_int64), ("valid_lo", C.c_int64),
                ("valid_hi", C.c_int64), ("trigger_capacity", C.c_int64), ("stream", C.c_void_p)]


class cui_tuning(C.Structure):
    _fields_ = [("n1", C.c_int32), ("ccols", C.c_int32), ("rpc", C.c_int32), ("batch", C.c_int32)]

    def as_dict(self):
        return {"n1": self.n1, "ccols": self.ccols, "rpc": self.rpc, "batch": self.batch}


class cui_trace_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("calls", C.c_int64), ("ms", C.c_double)]


PEAK_DTYPE = np.dtype([("sample", "<i8"), ("snr", "<f4"), ("phase", "<f4")])
TRIGGER_DTYPE = np.dtype([("tmpl", "<i4"), ("pad", "<i4"), ("sample", "<i8"), ("snr", "<f4"), ("phase", "<f4")])


class CuiError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load():
    """Load libcui.so (built by ``paper_1006_4644_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.cui_bank_create.argtypes = [C.POINTER(cui_bank_desc), vp, vp, C.c_int64, C.POINTER(vp)]
    lib.cui_segment_upload.argtypes = [vp, vp, C.c_int64, vp, C.c_int64, C.c_int]
    lib.cui_filter_bank.argtypes = [vp, vp, C.c_int64, vp]
    lib.cui_peaks.argtypes = [vp, vp, C.c_int64]
    lib.cui_triggers.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
    lib.cui_results.argtypes = [vp, vp, C.c_int64, vp, C.c_int64, C.POINTER(C.c_int64)]
    lib.cui_cluster_triggers.argtypes = [vp, vp, C.c_int64, C.POINTER(C.c_int64)]
    lib.cui_trigger_chisq.argtypes = [vp, C.c_int32, vp, C.c_int64, vp, vp]
    lib.cui_td_template.argtypes = [vp, C.c_int64, C.c_int32, vp, vp]
    lib.cui_bank_set_band.argtypes = [vp, C.c_double, C.c_double]
    lib.cui_band_correlate.argtypes = [vp, vp, vp, C.c_int64, C.c_double, C.c_double, vp, vp]
    lib.cui_band_combine.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_double, vp, vp, vp]
    lib.cui_template_bands.argtypes = [vp, vp, C.c_int64, C.c_int64, C.c_double, C.c_double, vp, vp]
    lib.cui_segment_band_series.argtypes = [vp, C.c_double, C.c_double, C.c_int32, vp]
    lib.cui_bank_sigma.argtypes = [vp, vp]
    lib.cui_bank_template.argtypes = [vp, C.c_int64, vp]
    lib.cui_bank_get_tuning.argtypes = [vp, C.POINTER(cui_tuning)]
    lib.cui_bank_set_tuning.argtypes = [vp, C.POINTER(cui_tuning)]
    lib.cui_bank_autotune.argtypes = [vp, C.c_int32, C.POINTER(cui_tuning), C.POINTER(C.c_double)]
    lib.cui_bank_set_wait_bounds.argtypes = [vp, C.c_int64, C.c_int64]
    lib.cui_template_sigma_noalloc.argtypes = [vp, C.c_int64, C.c_double, C.c_double, vp, vp, C.c_int64, vp, vp]
    lib.cui_template_sigma_noalloc.restype = C.c_int
    lib.cui_trace_enable.argtypes = [vp, C.c_int]
    lib.cui_trace_read.argtypes = [vp, C.POINTER(cui_trace_stat), C.c_int64, C.POINTER(C.c_int64)]
    lib.cui_bank_destroy.argtypes = [vp]
    lib.cui_bank_destroy.restype = None
    lib.cui_last_error.restype = C.c_char_p
    for name in ("cui_bank_create", "cui_segment_upload", "cui_filter_bank", "cui_peaks", "cui_triggers",
                 "cui_cluster_triggers", "cui_trigger_chisq", "cui_td_template", "cui_bank_set_band",
                 "cui_band_correlate", "cui_segment_band_series", "cui_results",
                 "cui_bank_sigma", "cui_bank_template", "cui_trace_enable", "cui_trace_read",
                 "cui_bank_get_tuning", "cui_bank_set_tuning", "cui_bank_autotune", "cui_bank_set_wait_bounds",
                 "cui_band_combine", "cui_template_bands"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def header_functions() -> list[str]:
    """Names of the functions include/cui.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cui_[a-z_0-9]+)\s*\(", text)))


def check(status: int, where: str):
    if status != CUI_OK:
        raise CuiError(status, where, load().cui_last_error().decode())
    return status


class cui_prescreen_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("sample_rate", C.c_double), ("f_low", C.c_double), ("bands", C.c_int32),
                ("frame", C.c_int32), ("regions", C.c_int32), ("max_batch", C.c_int32), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64),
                ("stream", C.c_void_p)]


def load_prescreen(lib):
    vp = C.c_void_p
    lib.cui_prescreen_create.argtypes = [C.POINTER(cui_prescreen_desc), C.POINTER(vp)]
    lib.cui_prescreen_destroy.argtypes = [vp]
    lib.cui_prescreen_destroy.restype = None
    lib.cui_prescreen_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    lib.cui_prescreen_features.argtypes = [vp, vp, vp, C.c_int64, vp]
    lib.cui_prescreen_bank_features.argtypes = [vp, vp, vp]
    lib.cui_prescreen_scores.argtypes = [vp, vp, C.c_int64, vp]
    lib.cui_prescreen_train_step.argtypes = [vp, vp, vp, C.c_int64, C.POINTER(C.c_float)]
    lib.cui_prescreen_gradient.argtypes = [vp, vp, vp, C.c_int64, vp, C.POINTER(C.c_float)]
    lib.cui_prescreen_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int64)]
    lib.cui_prescreen_set_state.argtypes = [vp, vp, vp, vp, C.c_int64]
    lib.cui_prescreen_rank.argtypes = [vp, vp, C.c_int64, vp, C.c_int32, C.c_int32, vp, C.POINTER(C.c_int64)]
    lib.cui_regions_create.argtypes = [vp, vp, C.c_int64, C.c_int32, C.POINTER(vp)]
    lib.cui_regions_order.argtypes = [vp, vp, C.c_int32, vp, C.POINTER(C.c_int64)]
    lib.cui_regions_destroy.argtypes = [vp]
    lib.cui_regions_destroy.restype = None
    lib.cui_prescreen_fit_norm.argtypes = [vp, vp, C.c_int64]
    lib.cui_prescreen_set_norm.argtypes = [vp, vp, vp]
    lib.cui_prescreen_get_norm.argtypes = [vp, vp, vp]
    lib.cui_prescreen_ensemble_scores.argtypes = [vp, C.c_int32, vp, C.c_int64, vp]
    for name in ("cui_prescreen_create", "cui_prescreen_info", "cui_prescreen_features", "cui_prescreen_bank_features",
                 "cui_prescreen_scores", "cui_prescreen_train_step", "cui_prescreen_gradient",
                 "cui_prescreen_get_state", "cui_prescreen_set_state", "cui_prescreen_rank",
                 "cui_prescreen_fit_norm", "cui_prescreen_set_norm", "cui_prescreen_get_norm",
                 "cui_prescreen_ensemble_scores", "cui_regions_create", "cui_regions_order"):
        getattr(lib, name).restype = C.c_int
    return lib
