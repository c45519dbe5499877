"""The chi^2 signal-consistency test on the GPU (cui_trigger_chisq) against
the oracle's FP64 definition at every trigger of a 64-template bank and at
sampled triggers of the 2^20-sample, 1024-template workload; the injected
template is signal-consistent; errors."""

import numpy as np
import pytest

import oracle
import synth
from parity import make_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()
    oracle.build()


def _check(w, dt, psd, trig, chi, rho, bands):
    m1, m2 = w.masses()
    for t in np.unique(trig["tmpl"]):
        sel = np.nonzero(trig["tmpl"] == t)[0]
        c_o, r_o = oracle.chisq(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n, trig["sample"][sel], bands)
        assert np.allclose(rho[sel], r_o, rtol=1e-3), (t, rho[sel], r_o)
        assert np.allclose(trig["snr"][sel], rho[sel], rtol=1e-4)  # the filter's generation method
        tol = 1e-3 * (c_o + 2 * bands) + 1e-4 * r_o ** 2
        assert np.all(np.abs(chi[sel] - c_o) <= tol), (t, chi[sel], c_o)


@pytest.mark.parametrize("bands", [4, 16])
def test_chisq_matches_the_oracle(bands):
    from paper_1006_4644_gb300 import Bank

    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, dt, (tmpl, j0, snr) = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=4.5, window=1024) as b:
        b.upload(strain, psd)
        b.filter()
        trig, _ = b.triggers()
        chi, rho = b.trigger_chisq(trig, bands)
    assert len(trig) > 10
    _check(w, dt, psd, trig, chi, rho, bands)
    # the injected template at the injection is signal-consistent: chi^2 ~ 2p - 2, far below rho^2
    hit = (trig["tmpl"] == tmpl[0]) & (np.abs(trig["sample"] - j0[0]) <= 1)
    assert hit.sum() == 1
    assert chi[hit][0] < 0.25 * rho[hit][0] ** 2


def test_chisq_at_2p20_sampled():
    from paper_1006_4644_gb300 import Bank

    w = synth.WORKLOADS["seg256s_bank1024_pn35"]
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.5) as b:
        b.upload(strain, psd)
        b.filter()
        trig, _ = b.triggers()
        pick = trig[np.random.default_rng(1).permutation(len(trig))[:12]]
        chi, rho = b.trigger_chisq(pick, 16)
    _check(w, dt, psd, pick, chi, rho, 16)


def test_chisq_errors():
    from paper_1006_4644_gb300 import CUI_PLAIN, TRIGGER_DTYPE, Bank, CuiError, _lib

    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, _, _ = make_segment(w)
    m1, m2 = w.masses()
    kw = dict(n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0)
    with Bank(m1, m2, **kw) as b:
        rec = np.zeros(1, dtype=TRIGGER_DTYPE)
        with pytest.raises(CuiError) as e:
            b.trigger_chisq(rec, 16)
        assert e.value.status == _lib.CUI_ERR_STATE  # no segment
        b.upload(strain, psd)
        for bands in (0, 65):
            with pytest.raises(CuiError) as e:
                b.trigger_chisq(rec, bands)
            assert e.value.status == _lib.CUI_ERR_ARG
        bad = rec.copy()
        bad["sample"] = w.n
        with pytest.raises(CuiError) as e:
            b.trigger_chisq(bad, 16)
        assert e.value.status == _lib.CUI_ERR_ARG
        assert len(b.trigger_chisq(rec[:0], 16)[0]) == 0
    with Bank(m1, m2, flags=CUI_PLAIN, **kw) as b:
        b.upload(strain, psd)
        with pytest.raises(CuiError) as e:
            b.trigger_chisq(rec, 16)
        assert e.value.status == _lib.CUI_ERR_STATE


def test_post_filter_sums_do_not_depend_on_the_filter_tiling():
    """chi^2 and the band correlators use their own anchor tables (one anchor
    per 32 bins), so for the same triggers and queries their results are the
    same bit for bit whether the filter runs on 16 or 32 columns per pass-1
    CTA."""
    from paper_1006_4644_gb300 import Bank

    w = synth.WORKLOADS["seg256s_bank1024_pn35"]
    strain, psd, _, _ = make_segment(w)
    m1, m2 = w.masses()
    m1, m2 = m1[:64], m2[:64]
    tm = np.arange(0, 64, 5, dtype=np.int32)
    ts = 0.37 * tm + 1.5
    pick, out = None, []
    for ccols in (16, 32):
        with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0) as b:
            b.upload(strain, psd)
            b.set_tuning(256, ccols, 0, 64)
            if pick is None:
                b.filter()
                trig, _ = b.triggers()
                pick = trig[:32]
            chi, rho = b.trigger_chisq(pick, 16)
            z, s2 = b.band_correlate(tm, ts, 0.0, 80.0)
            out.append((chi, rho, z, s2))
    assert len(pick) > 0
    for a, b_ in zip(out[0], out[1]):
        assert np.array_equal(a, b_)
