"""Multi-band search on the GPU: the band-limited filter (cui_bank_set_band)
against the oracle's band filter; the band correlators at arbitrary times
(cui_band_correlate) against the oracle's direct sums and against the filter's
own peaks, at 2^16 and sampled at 2^20; the band filter sampled at 2^20; the
band-limited, resampled series (cui_segment_band_series) against the oracle's at
2^16 and 2^20; and the hierarchical search recovering a chirp that is longer
than the short segments its upper band is searched on."""

import math

import numpy as np
import pytest

import oracle
import synth
from parity import Report, check_template, make_segment, split_triggers

pytestmark = pytest.mark.gpu

W16 = synth.WORKLOADS["seg16s_bank64_pn2"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()
    oracle.build()


def _bank(w, **kw):
    from paper_1006_4644_gb300 import Bank

    m1, m2 = w.masses()
    return Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, **kw)


@pytest.mark.parametrize("band,plain", [((60.0, 0.0), False), ((45.0, 150.0), False), ((60.0, 0.0), True)])
def test_band_filter_matches_the_oracle(band, plain):
    from paper_1006_4644_gb300 import CUI_PLAIN

    w = W16
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    thr = 4.5
    with _bank(w, snr_threshold=thr, flags=CUI_PLAIN if plain else 0) as b:
        b.upload(strain, psd)
        b.filter()
        full = b.peaks()
        b.set_band(*band)
        b.filter()
        peaks, (trig, _), sig = b.peaks(), b.triggers(), b.sigma()
        b.set_band()  # the full band again: the same result as before
        b.filter()
        again = b.peaks()
    assert np.array_equal(again, full)
    per = split_triggers(trig, w.n_templates)
    rep = Report()
    for t in range(w.n_templates):
        h, _, _ = oracle.spa_template(m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
        ka, kb = oracle.band_edges(m1[t], m2[t], w.f_low, w.fs, w.n, *band)
        s2 = oracle.sigma2(h, psd, w.fs, w.n, ka, kb)
        assert abs(sig[t] - math.sqrt(s2)) <= 1e-9 * math.sqrt(s2)
        z = oracle.correlate(dt, h, psd, w.fs, w.n, ka, kb)
        check_template(rep, t, z, np.abs(z) ** 2 / s2, peaks[t], per[t], 0, w.n, int(w.fs), thr)
    assert not rep.errors, rep.errors[:5]
    assert len(trig) > 0


def test_band_filter_at_2p20_sampled():
    """The band-limited filter at the full size of the 1024-template, 2^20-sample
    workload (its own tiling), against the oracle's band filter on sampled
    templates, including the injected ones."""
    w = synth.WORKLOADS["seg256s_bank1024_pn35"]
    strain, psd, dt, (tmpl, _, _) = make_segment(w)
    m1, m2 = w.masses()
    band, thr = (80.0, 0.0), 5.5
    with _bank(w, snr_threshold=thr) as b:
        b.upload(strain, psd)
        b.set_band(*band)
        b.filter()
        peaks, (trig, _), sig = b.peaks(), b.triggers(), b.sigma()
    per = split_triggers(trig, w.n_templates)
    pick = sorted(set(int(t) for t in tmpl) | set(np.random.default_rng(3).integers(0, w.n_templates, 8).tolist()))
    rep = Report()
    for t in pick:
        h, _, _ = oracle.spa_template(m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
        ka, kb = oracle.band_edges(m1[t], m2[t], w.f_low, w.fs, w.n, *band)
        s2 = oracle.sigma2(h, psd, w.fs, w.n, ka, kb)
        assert abs(sig[t] - math.sqrt(s2)) <= 1e-9 * math.sqrt(s2)
        z = oracle.correlate(dt, h, psd, w.fs, w.n, ka, kb)
        check_template(rep, t, z, np.abs(z) ** 2 / s2, peaks[t], per[t], 0, w.n, int(w.fs), thr)
    assert not rep.errors, rep.errors[:5]


def test_band_combine_matches_the_oracle():
    """cui_band_combine: the upper band on one bank and the lower band on
    another, added coherently in the library, against the oracle's direct band
    sums combined as rho = |z_h + z_l| / sqrt(sigma_h^2 + sigma_l^2); with both
    banks on the same segment and time, the split bands make up the full band,
    so rho is the filter's own peak; its per-band sums are those
    cui_band_correlate returns."""
    from paper_1006_4644_gb300 import Bank, CuiError, _lib

    w = W16
    strain, psd, dt, (tmpl, j0, _) = make_segment(w)
    m1, m2 = w.masses()
    f_split = 70.0
    with _bank(w) as hb, _bank(w) as lb:
        hb.upload(strain, psd)
        lb.upload(strain, psd)
        hb.filter()
        pk = hb.peaks()
        tm = np.unique(np.concatenate([np.arange(0, w.n_templates, 5), tmpl])).astype(np.int32)
        ts = pk["sample"][tm] / w.fs
        rho, ph, sums = hb.band_combine(ts, lb, ts, tm, f_split)
        zh, s2h = hb.band_correlate(tm, ts, f_split, 0.0)
        zl, s2l = lb.band_correlate(tm, ts, 0.0, f_split)
        assert np.array_equal(sums[:, 0] + 1j * sums[:, 1], zh) and np.array_equal(sums[:, 2], s2h)
        assert np.array_equal(sums[:, 3] + 1j * sums[:, 4], zl) and np.array_equal(sums[:, 5], s2l)
        assert np.max(np.abs(rho / pk["snr"][tm] - 1.0)) < 1e-3
        with pytest.raises(CuiError) as e:
            hb.band_combine(ts, lb, ts, tm, 0.0)
        assert e.value.status == _lib.CUI_ERR_ARG
        with Bank(m1[::-1].copy(), m2[::-1].copy(), n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2) as other:
            other.upload(strain, psd)
            with pytest.raises(CuiError) as e:
                hb.band_combine(ts, other, ts, tm, f_split)
            assert e.value.status == _lib.CUI_ERR_ARG
    for i, t in enumerate(tm):
        a, sa = oracle.band_correlate(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n, [ts[i]], f_split, 0.0)
        b, sb = oracle.band_correlate(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n, [ts[i]], 0.0, f_split)
        z = a[0] + b[0]
        want = abs(z) / math.sqrt(sa + sb)
        assert abs(rho[i] - want) <= 1e-3 * want, (t, rho[i], want)
        assert abs((ph[i] - np.angle(z) + math.pi) % (2 * math.pi) - math.pi) < 2e-3


@pytest.mark.parametrize("ccols", [16, 32, 64])
def test_band_correlate_matches_the_oracle(ccols):
    """Bins are generated in blocks of `ccols` (the pass-1 tiling), so every
    block width is checked."""
    w = W16
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    rng = np.random.default_rng(5)
    tm = rng.integers(0, w.n_templates, 24).astype(np.int32)
    # sample times, and arbitrary ones (before the segment and past its end wrap)
    ts = np.concatenate([rng.integers(0, w.n, 12) / w.fs, rng.uniform(-3.0, 20.0, 12)])
    worst = 0.0
    with _bank(w) as b:
        b.upload(strain, psd)
        b.set_tuning(64, ccols, 4, w.n_templates)
        b.set_band(100.0, 0.0)  # the filter's band does not change the band sums
        for band in ((0.0, 0.0), (0.0, 80.0), (80.0, 0.0), (55.5, 300.0)):
            z, s2 = b.band_correlate(tm, ts, *band)
            for i in range(len(tm)):
                t = int(tm[i])
                zo, so = oracle.band_correlate(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n, [ts[i]], *band)
                assert abs(s2[i] - so) <= 1e-9 * so
                sg = math.sqrt(so)
                err = abs(z[i] - zo[0]) / (sg * max(1.0, abs(zo[0]) / sg))
                worst = max(worst, err)
        assert worst < 1e-3, worst
        # at the filter's peaks, over the filter's band: the filter's rho and phase
        b.set_band()
        b.filter()
        pk = b.peaks()
        z, s2 = b.band_correlate(np.arange(w.n_templates), pk["sample"] / w.fs)
    rho = np.abs(z) / np.sqrt(s2)
    assert np.allclose(rho, pk["snr"], rtol=2e-4)
    dphi = np.angle(np.exp(1j * (np.angle(z) - pk["phase"])))
    assert np.max(np.abs(dphi)) < 2e-3


def test_band_correlate_at_2p20_sampled():
    w = synth.WORKLOADS["seg256s_bank1024_pn35"]
    strain, psd, dt, (tmpl, j0, _) = make_segment(w)
    m1, m2 = w.masses()
    rng = np.random.default_rng(9)
    tm = np.concatenate([tmpl[:3], rng.integers(0, w.n_templates, 5)]).astype(np.int32)
    ts = np.concatenate([j0[:3] / w.fs, rng.uniform(0.0, w.n / w.fs, 5)])
    with _bank(w) as b:
        b.upload(strain, psd)
        z, s2 = b.band_correlate(tm, ts, 0.0, 100.0)
    for i in range(len(tm)):
        t = int(tm[i])
        zo, so = oracle.band_correlate(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n, [ts[i]], 0.0, 100.0)
        assert abs(s2[i] - so) <= 1e-9 * so
        sg = math.sqrt(so)
        assert abs(z[i] - zo[0]) <= 1e-3 * sg * max(1.0, abs(zo[0]) / sg), (i, z[i], zo[0])


@pytest.mark.parametrize("band,decim,wname", [((60.0, 0.0), 1, "seg16s_bank64_pn2"), ((0.0, 60.0), 8, "seg16s_bank64_pn2"),
                                              ((20.0, 300.0), 4, "seg16s_bank64_pn2"),
                                              ((40.0, 0.0), 1, "seg256s_bank1024_pn35"),
                                              ((0.0, 40.0), 8, "seg256s_bank1024_pn35")])
def test_band_series_matches_the_oracle(band, decim, wname):
    import torch

    w = synth.WORKLOADS[wname]
    strain, psd, _, _ = make_segment(w)
    with _bank(w) as b:
        b.upload(strain, psd)
        out = torch.empty(w.n // decim, dtype=torch.float64, device="cuda")
        b.band_series(out, *band, decim)
        got = out.cpu().numpy()
    want = oracle.band_series(strain, w.fs, *band, decim)
    assert np.max(np.abs(got - want)) <= 1e-9 * np.max(np.abs(strain))


def test_band_calls_reject_bad_arguments():
    import torch

    from paper_1006_4644_gb300 import CuiError

    w = W16
    strain, psd, _, _ = make_segment(w)
    with _bank(w) as b:
        with pytest.raises(CuiError):  # no segment yet
            b.band_correlate([0], [0.0])
        b.upload(strain, psd)
        with pytest.raises(CuiError):
            b.band_correlate([w.n_templates], [0.0])
        with pytest.raises(CuiError):
            b.band_correlate([0], [float("nan")])
        with pytest.raises(CuiError):
            b.set_band(float("inf"), 0.0)
        out = torch.empty(w.n // 3, dtype=torch.float64, device="cuda")
        with pytest.raises((CuiError, ValueError)):
            b.band_series(out, 0.0, 0.0, 3)


def test_hierarchical_search_recovers_a_long_chirp():
    """A 1.4 + 1.4 solar-mass chirp from 20 Hz lasts about 160 s; the upper
    band from 60 Hz lasts about 8 s and is searched on 16 s segments.  The
    detection is completed by the lower band, summed on the whole 256 s
    segment or on its lower band decimated to 512 Hz."""
    import torch

    from paper_1006_4644_gb300 import Bank
    from paper_1006_4644_gb300.multiband import hierarchical_search

    n, fs, f_low, pn, f_split = 1 << 20, 4096.0, 20.0, 7, 60.0
    ns, decim = 1 << 16, 8
    r1, r2 = synth.sample_masses(1006_4650, 1, 7, 1.0, 3.0, False)
    m1 = np.concatenate([[1.4], r1])
    m2 = np.concatenate([[1.4], r2])
    psd = synth.psd_onesided(n, fs)
    d = synth.noise_spectrum(1006_4650, 2, n, fs, psd, f_low)
    h, k_lo, k_hi = oracle.spa_template(m1[0], m2[0], pn, f_low, fs, n)
    j0 = 200 * 4096 + 123
    synth.add_signal(d, h, 15.0 / math.sqrt(oracle.sigma2(h, psd, fs, n, k_lo, k_hi)), j0, n)
    strain = synth.strain_from_spectrum(d, n, fs)
    dt = oracle.segment_spectrum(strain, fs)

    def dev(x):
        x = np.array(x, dtype=np.float64)
        x[0] = 1.0
        return torch.from_numpy(x).cuda()

    kw = dict(f_low=f_low, pn_x2=pn)
    with Bank(m1, m2, n=n, fs=fs, **kw) as seg, \
            Bank(m1, m2, n=ns, fs=fs, snr_threshold=8.0, valid=(40960, 61440), **kw) as det, \
            Bank(m1, m2, n=n // decim, fs=fs / decim, **kw) as low:
        seg.upload(torch.from_numpy(strain).cuda(), dev(psd))
        lows = torch.empty(n // decim, dtype=torch.float64, device="cuda")
        seg.band_series(lows, 0.0, f_split, decim)
        low.upload(lows, dev(psd[: n // decim // 2 + 1]))
        psd_s = dev(synth.psd_onesided(ns, fs))
        cand = hierarchical_search(seg, det, f_split, psd_s)
        cand_dec = hierarchical_search(seg, det, f_split, psd_s, low=low)
        assert len(cand) > 0
        # every detection is the injection, by one template or another
        assert np.all(np.abs(cand["t"] - j0 / fs) < 2.0)
        best = cand[np.argmax(np.where(cand["tmpl"] == 0, cand["rho"], -1.0))]
        assert best["tmpl"] == 0 and abs(best["t"] * fs - j0) <= 2
        # the full band on the whole segment at the detection
        zf, sf = seg.band_correlate([0], [best["t"]])
    rho_full = abs(zf[0]) / math.sqrt(sf[0])
    zo, so = oracle.band_correlate(dt, psd, m1[0], m2[0], pn, f_low, fs, n, [best["t"]], 0.0, 0.0)
    rho_o = abs(zo[0]) / math.sqrt(so)
    assert abs(rho_full - rho_o) <= 1e-3 * rho_o
    assert abs(best["rho"] - rho_full) <= 1e-2 * rho_full
    assert rho_full > 12.0
    # the decimated lower band gives the same combination
    assert np.array_equal(cand_dec["tmpl"], cand["tmpl"]) and np.array_equal(cand_dec["t"], cand["t"])
    assert np.allclose(cand_dec["rho"], cand["rho"], rtol=1e-3)
