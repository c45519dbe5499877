"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the
same seeded inputs (rules in tests/parity.py: sample indices exact unless the
oracle itself has a near tie, rho within 1e-3 relative, phase within 2e-3 rad).
"""

import math

import numpy as np
import pytest

import oracle
import synth
from parity import compare_bank, make_segment, oracle_series

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()
    oracle.build()


def _bank(w, flags=0, thr=6.0, window=None, valid=(0, None), m=None, cap=0):
    from paper_1006_4644_gb300 import Bank

    m1, m2 = w.masses() if m is None else m
    return Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, flags=flags, snr_threshold=thr,
                window=window, valid=valid, trigger_capacity=cap)


def _run(w, strain, psd, flags=0, thr=6.0, window=None, valid=(0, None), order=None):
    with _bank(w, flags, thr, window, valid) as b:
        b.upload(strain, psd)
        b.filter(order)
        return b.peaks(), b.triggers()[0], b.sigma()


W1 = synth.WORKLOADS["seg16s_bank64_pn2"]


@pytest.fixture(scope="module")
def seg16s():
    return make_segment(W1)


@pytest.mark.parametrize("flags", [0, 1, 4, 12], ids=["fused_df", "fused_fp64", "plain_fp32", "plain_fp64"])
def test_seg16s_bank64_all_paths(seg16s, flags):
    from paper_1006_4644_gb300 import CUI_PLAIN

    strain, psd, dt, (tmpl, j0, snr) = seg16s
    peaks, trig, sig = _run(W1, strain, psd, flags)
    rep = compare_bank(W1, dt, psd, peaks, trig, range(W1.n_templates), 0, W1.n, int(W1.fs), 6.0)
    assert rep.ok(), rep
    assert rep.ambiguous <= 2, rep
    # sigma against the oracle's normalisation
    m1, m2 = W1.masses()
    for t in range(0, W1.n_templates, 7):
        h, lo, hi = oracle.spa_template(m1[t], m2[t], W1.pn_x2, W1.f_low, W1.fs, W1.n)
        s2 = oracle.sigma2(h, psd, W1.fs, W1.n, lo, hi)
        tol = 1e-6 if (flags & CUI_PLAIN) and not (flags & 8) else 1e-10
        assert abs(sig[t] / math.sqrt(s2) - 1) < tol
    # the injection is found where it was put
    t = int(tmpl[0])
    assert abs(int(peaks[t]["sample"]) - int(j0[0])) <= 1
    assert 9.0 < peaks[t]["snr"] < 15.0


@pytest.mark.parametrize("log2n", [12, 13, 14, 15, 17, 18, 19])
@pytest.mark.parametrize("fp64_anchor", [False, True])
def test_tiling_sizes_with_ragged_windows(log2n, fp64_anchor):
    n = 1 << log2n
    w = synth.Workload(f"n{log2n}", n, 4096.0, 30.0 if log2n >= 14 else 60.0, 7, 6, 1.0, 6.0, False, 1, 20.0,
                       20.0, 1.0, 777 + log2n)
    strain, psd, dt, plan = make_segment(w)
    lo, hi, window = n // 8, n - n // 5, 1000 if n > 4000 else 333
    peaks, trig, _ = _run(w, strain, psd, 1 if fp64_anchor else 0, thr=5.0, window=window, valid=(lo, hi))
    rep = compare_bank(w, dt, psd, peaks, trig, range(w.n_templates), lo, hi, window, 5.0)
    assert rep.ok(), rep


W2 = synth.WORKLOADS["seg256s_bank1024_pn35"]


@pytest.fixture(scope="module")
def seg256s():
    return make_segment(W2)


@pytest.mark.parametrize("tuning", [None, (256, 16, 0, 256)], ids=["default", "bench"])
def test_seg256s_bank1024_fused_full(seg256s, tuning):
    """The whole metric workload, in the default tiling and in the one the
    benchmark's autotuner picks on GB300 (streamed pass 2, batches of 256)."""
    strain, psd, dt, (tmpl, j0, snr) = seg256s
    with _bank(W2) as b:
        b.upload(strain, psd)
        if tuning:
            b.set_tuning(*tuning)
        b.filter()
        peaks, trig = b.peaks(), b.triggers()[0]
    rep = compare_bank(W2, dt, psd, peaks, trig, range(W2.n_templates), 0, W2.n, int(W2.fs), 6.0)
    assert rep.ok(), rep
    assert rep.ambiguous <= 10, rep
    # each injected template triggers at its injection with about its SNR
    for t, j, s in zip(tmpl, j0, snr):
        near = trig[(trig["tmpl"] == t) & (np.abs(trig["sample"] - int(j)) <= 2)]
        assert len(near) == 1, (t, j)
        assert abs(float(near["snr"][0]) - s) < 3.5


def test_seg256s_plain_fp32_subset(seg256s):
    from paper_1006_4644_gb300 import CUI_PLAIN

    strain, psd, dt, (tmpl, j0, snr) = seg256s
    order = np.unique(np.concatenate([np.arange(0, W2.n_templates, 97), tmpl]))
    peaks, trig, _ = _run(W2, strain, psd, CUI_PLAIN, order=order)
    rep = compare_bank(W2, dt, psd, peaks, trig, order, 0, W2.n, int(W2.fs), 6.0)
    assert rep.ok(), rep


def test_seg1024s_bank10k_sampled():
    w = synth.WORKLOADS["seg1024s_bank10k_pn35"]
    strain, psd, dt, (tmpl, j0, snr) = make_segment(w)
    peaks, trig, _ = _run(w, strain, psd, 0)
    rng = np.random.default_rng(3)
    sample = np.unique(np.concatenate([rng.choice(w.n_templates, 20, replace=False), tmpl]))
    rep = compare_bank(w, dt, psd, peaks, trig, sample, 0, w.n, int(w.fs), 6.0)
    assert rep.ok(), rep
    # properties that hold for every template: rho >= 0, samples in range
    assert np.all(peaks["snr"] >= 0) and np.all((peaks["sample"] >= 0) & (peaks["sample"] < w.n))


def test_template_readout_mismatch():
    """Mismatch Delta = 1 - <h_cpu, h_gpu> / <h_cpu, h_cpu> (eq:mismatch) of the
    fused generator's template against the oracle's."""
    import torch

    w = W2
    m1, m2 = w.masses()
    psd = w.psd()
    with _bank(w) as b:
        out = torch.zeros(w.n // 2 + 1, dtype=torch.complex64, device="cuda")
        worst = 0.0
        for t in range(0, w.n_templates, 64):
            b.template(t, out)
            hg = out.cpu().numpy().astype(np.complex128)
            ho, lo, hi = oracle.spa_template(m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
            k = slice(lo, hi)
            inner = lambda a, c: 4 * w.df * np.sum(a[k] * np.conj(c[k]) / psd[k]).real
            delta = 1 - inner(ho, hg) / inner(ho, ho)
            worst = max(worst, abs(delta))
        assert worst < 1e-6, worst


def test_device_upload_matches_host_upload(seg16s):
    import torch

    strain, psd, dt, _ = seg16s
    a = _run(W1, strain, psd, 0)
    ps = psd.copy()
    ps[0] = 1.0  # bin 0 is never read; keep the device copy finite
    with _bank(W1) as b:
        b.upload(torch.from_numpy(strain).cuda(), torch.from_numpy(ps).cuda())
        b.filter()
        p = b.peaks()
    assert np.array_equal(a[0]["sample"], p["sample"]) and np.array_equal(a[0]["snr"], p["snr"])


@pytest.mark.parametrize("wname,count", [("seg16s_bank64_pn2", 64), ("seg256s_bank1024_pn35", 24),
                                         ("seg1024s_bank10k_pn35", 6)])
def test_bf16_storage_within_its_bound(wname, count):
    """CUI_STORE_BF16 keeps Y (the spectrum between the FFT passes) as bf16
    pairs: each value rounds to 2^-9 relative, so rho may move by a few 1e-3.
    Against the FP64 oracle: every peak rho within 5e-3 relative, and every
    peak sample exact unless the oracle's rho at the reported sample is within
    5e-3 of its maximum.  At 2^20 this runs the streamed pass 2 (both teams)
    with bf16 row pairs in its staging buffer; at 2^22 the split pass 2 with
    the bf16 row halves in its staging buffer and team 0's exchange buffer."""
    from paper_1006_4644_gb300 import CUI_STORE_BF16

    w = synth.WORKLOADS[wname]
    strain, psd, dt, (tmpl, _, _) = make_segment(w)
    m1, m2 = w.masses()
    order = np.unique(np.concatenate([np.arange(count), tmpl])).astype(np.int32)
    with _bank(w, CUI_STORE_BF16) as b:
        b.upload(strain, psd)
        if w.n >= 1 << 20:
            assert b.tuning()["rpc"] == 0  # the default tiling at 2^20 and 2^22 is the streamed pass 2
        b.filter(order)
        peaks = b.peaks()
    worst = 0.0
    for t in order:
        z, r2, _ = oracle_series(dt, psd, m1[t], m2[t], w.pn_x2, w.f_low, w.fs, w.n)
        j = int(np.argmax(r2))
        got = float(peaks[t]["snr"])
        rel = abs(got - math.sqrt(r2[j])) / math.sqrt(r2[j])
        worst = max(worst, rel)
        assert rel < 5e-3, (t, got, math.sqrt(r2[j]))
        s = int(peaks[t]["sample"])
        assert s == j or math.sqrt(r2[s] / r2[j]) >= 1 - 5e-3, (t, s, j)
    print(f"bf16 storage: max relative SNR error {worst:.2e} over {len(order)} templates")
