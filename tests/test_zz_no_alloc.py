"""The allocation-free normalisation entry point (GPU).

Some callers cannot allocate device memory when they need a result (a
pool-owned memory budget, a real-time loop that cannot wait for cudaMalloc);
cui_template_sigma_noalloc serves them with scratch compiled into the
library.  Its sigma^2 must equal what cui_bank_sigma gives for the same bank
and PSD, on two calls in a row (the second call finds the previous call's
contents in the shared scratch).  This file is collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["seg16s_bank64_pn2", "seg256s_bank1024_pn35"])
def test_noalloc_sigma_matches_bank_sigma_twice(name):
    import torch

    from paper_1006_4644_gb300 import Bank, _lib, build

    build.build()
    lib = _lib.load()
    w = synth.WORKLOADS[name]
    m1, m2 = w.masses()
    psd = w.psd()
    psd_fin = psd.copy()
    psd_fin[0] = 1.0  # bin 0 is never read
    strain = synth.strain_from_spectrum(w.noise(), w.n, w.fs)
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2) as b:
        b.upload(strain, psd)
        ref = b.sigma()
    psd_d = torch.from_numpy(psd_fin).cuda()
    stream = torch.cuda.current_stream()
    m1c = np.ascontiguousarray(m1)
    m2c = np.ascontiguousarray(m2)
    for call in range(2):
        out = torch.full((w.n_templates,), -1.0, dtype=torch.float64, device="cuda")
        st = lib.cui_template_sigma_noalloc(psd_d.data_ptr(), w.n, w.fs, w.f_low, m1c.ctypes.data, m2c.ctypes.data,
                                            w.n_templates, out.data_ptr(), stream.cuda_stream)
        assert st == _lib.CUI_OK, lib.cui_last_error()
        torch.cuda.synchronize()
        got = np.sqrt(out.cpu().numpy())
        assert np.max(np.abs(got / ref - 1.0)) < 1e-12, (call, np.max(np.abs(got / ref - 1.0)))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    from paper_1006_4644_gb300 import _lib, build

    build.build()
    lib = _lib.load()
    psd_d = torch.ones((1 << 21) + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    m = np.full(4, 1.4)
    st = lib.cui_template_sigma_noalloc(psd_d.data_ptr(), 1 << 22, 4096.0, 20.0, m.ctypes.data, m.ctypes.data, 4,
                                        out.data_ptr(), None)
    assert st == _lib.CUI_ERR_ARG and b"allocation-free maximum" in lib.cui_last_error()
    big = np.full(20000, 1.4)
    st = lib.cui_template_sigma_noalloc(psd_d.data_ptr(), 1 << 16, 4096.0, 20.0, big.ctypes.data, big.ctypes.data,
                                        len(big), out.data_ptr(), None)
    assert st == _lib.CUI_ERR_ARG and b"allocation-free maximum" in lib.cui_last_error()
