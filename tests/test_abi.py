"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/cui.h declares (no compute calls here)."""

import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1006_4644_gb300 import _lib, build

    build.build()
    return _lib.load()


def test_exports_every_declared_function(lib):
    from paper_1006_4644_gb300 import _lib

    names = _lib.header_functions()
    assert {"cui_bank_create", "cui_segment_upload", "cui_filter_bank", "cui_triggers"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(lib):
    from paper_1006_4644_gb300 import _lib

    assert ctypes.sizeof(_lib.cui_bank_desc) == 88
    assert _lib.PEAK_DTYPE.itemsize == 16
    assert _lib.TRIGGER_DTYPE.itemsize == 24


def test_argument_errors_need_no_gpu(lib):
    # argument validation happens before any CUDA call
    from paper_1006_4644_gb300 import _lib

    d = _lib.cui_bank_desc()
    d.n, d.sample_rate, d.f_low, d.pn_order_x2, d.window = 1000, 4096.0, 30.0, 7, 4096
    h = ctypes.c_void_p()
    m = (ctypes.c_double * 1)(1.4)
    st = lib.cui_bank_create(ctypes.byref(d), ctypes.addressof(m), ctypes.addressof(m), 1, ctypes.byref(h))
    assert st == _lib.CUI_ERR_ARG and b"power of two" in lib.cui_last_error()
    assert h.value is None
    st = lib.cui_filter_bank(None, None, 0, None)
    assert st == _lib.CUI_ERR_ARG


def test_prescreen_create_rejects_bad_rates_without_a_gpu(lib):
    # the band edges are cast to integers only after the rate and f_low are checked
    from paper_1006_4644_gb300 import _lib

    _lib.load_prescreen(lib)
    h = ctypes.c_void_p()
    for fs, f_low in ((float("inf"), 30.0), (float("nan"), 30.0), (4096.0, 2048.0), (4096.0, 1e300), (4096.0, 0.0)):
        d = _lib.cui_prescreen_desc(n=1 << 16, sample_rate=fs, f_low=f_low, bands=16, frame=512, regions=100,
                                    max_batch=64, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=1)
        st = lib.cui_prescreen_create(ctypes.byref(d), ctypes.byref(h))
        assert st == _lib.CUI_ERR_ARG and b"f_low" in lib.cui_last_error(), (fs, f_low)
        assert h.value is None
