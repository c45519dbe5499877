"""Edge cases and error statuses through the C ABI (GPU)."""

import numpy as np
import pytest

import oracle
import synth
from parity import compare_bank, make_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()


W = synth.Workload("edge", 1 << 14, 4096.0, 30.0, 7, 6, 1.0, 4.0, False, 1, 25.0, 25.0, 1.0, 4242)


@pytest.fixture(scope="module")
def seg():
    return make_segment(W)


def _bank(**kw):
    from paper_1006_4644_gb300 import Bank

    m1, m2 = kw.pop("m", W.masses())
    args = dict(n=W.n, fs=W.fs, f_low=W.f_low, pn_x2=W.pn_x2)
    args.update(kw)
    return Bank(m1, m2, **args)


@pytest.mark.parametrize("flags", [0, 4])
def test_empty_band_templates(seg, flags):
    strain, psd, _, _ = seg
    m = (np.array([80.0, 1.5]), np.array([80.0, 1.5]))  # f_ISCO(160 Msun) < f_low
    with _bank(m=m, flags=flags) as b:
        b.upload(strain, psd)
        b.filter()
        p = b.peaks()
        s = b.sigma()
        tr, tot = b.triggers()
    assert s[0] == 0 and p[0]["snr"] == 0 and p[0]["sample"] == 0
    assert s[1] > 0 and p[1]["snr"] > 0
    assert not np.any(tr["tmpl"] == 0)


def test_empty_valid_range(seg):
    strain, psd, _, _ = seg
    with _bank(valid=(100, 100)) as b:
        b.upload(strain, psd)
        b.filter()
        p = b.peaks()
        tr, tot = b.triggers()
    assert tot == 0 and np.all(p["sample"] == 100) and np.all(p["snr"] == 0)


def test_zero_threshold_overflow_and_exact_count(seg):
    from paper_1006_4644_gb300 import CuiError, _lib

    strain, psd, _, _ = seg
    nwin = -(-W.n // 1000)
    with _bank(snr_threshold=0.0, window=1000) as b:
        b.upload(strain, psd)
        b.filter()
        tr, tot = b.triggers()
        assert tot == W.n_templates * nwin and len(tr) == tot
        small, tot2 = b.triggers(capacity=5, allow_overflow=True)
        assert tot2 == tot and len(small) == 5
        with pytest.raises(CuiError) as e:
            b.triggers(capacity=5)
        assert e.value.status == _lib.CUI_ERR_OVERFLOW
    # a device buffer smaller than the total: overflow, peaks still right
    with _bank(snr_threshold=0.0, window=1000, trigger_capacity=7) as b:
        b.upload(strain, psd)
        b.filter()
        tr, tot = b.triggers(allow_overflow=True)
        assert tot == W.n_templates * nwin and len(tr) == 7
        with _bank() as ref:
            ref.upload(strain, psd)
            ref.filter()
            assert np.array_equal(ref.peaks()["sample"], b.peaks()["sample"])


def test_order_subset_and_repeat_calls(seg):
    strain, psd, dt, _ = seg
    with _bank(snr_threshold=4.0) as b:
        b.upload(strain, psd)
        b.filter()
        full = b.peaks()
        tr_full, _ = b.triggers()
        b.filter(order=[4, 1])
        sub = b.peaks()
        tr_sub, _ = b.triggers()
    assert np.array_equal(sub[[1, 4]], full[[1, 4]])
    assert set(tr_sub["tmpl"].tolist()) <= {1, 4}
    assert len(tr_sub) == int(np.sum(np.isin(tr_full["tmpl"], [1, 4])))


def test_error_statuses(seg):
    from paper_1006_4644_gb300 import CuiError, _lib

    strain, psd, _, _ = seg
    with _bank() as b:
        with pytest.raises(CuiError) as e:
            b.filter()
        assert e.value.status == _lib.CUI_ERR_STATE
        with pytest.raises(CuiError) as e:
            b.upload(strain[:-2], psd)
        assert e.value.status == _lib.CUI_ERR_ARG
        bad = psd.copy()
        bad[W.n // 4] = -1.0
        with pytest.raises(CuiError) as e:
            b.upload(strain, bad)
        assert e.value.status == _lib.CUI_ERR_ARG
        b.upload(strain, psd)
        with pytest.raises(CuiError) as e:
            b.filter(order=[0, W.n_templates])
        assert e.value.status == _lib.CUI_ERR_ARG
        with pytest.raises(CuiError) as e:
            b.filter(order=[1, 1])
        assert e.value.status == _lib.CUI_ERR_ARG
    with pytest.raises(CuiError) as e:
        _bank(n=3000)
    assert e.value.status == _lib.CUI_ERR_ARG
    with pytest.raises(CuiError):
        _bank(m=(np.array([1.0, -1.0]), np.array([1.0, 1.0])))


@pytest.mark.parametrize("case", ["fused_rounds0", "fused_rounds1_contended", "plain_rounds0", "streamed_wait0",
                                  "streamed16k_wait0"])
def test_bounded_waits_report_a_timeout_and_the_handle_recovers(case):
    """The device waits are bounded and a wait that runs out is reported, not
    hung on.  cui_bank_set_wait_bounds lowers the bounds: no round of the
    compare-and-swap loops that raise the peak and window slots (every update
    gives up), a single round under a zero threshold (thousands of samples
    race for each window slot, so updates that lose a race give up), or a zero
    time limit for the streamed pass 2's wait for its row pair (each team gives
    up on its first row pair; the copy in flight still lands before the CTA
    exits).  The next read-out returns CUI_ERR_TIMEOUT; with the defaults back,
    a new upload and filter match the oracle again on the same handle."""
    from paper_1006_4644_gb300 import CUI_PLAIN, CuiError, _lib

    if case == "streamed_wait0":
        w = synth.Workload("edge18", 1 << 18, 4096.0, 30.0, 7, 4, 1.0, 6.0, False, 1, 25.0, 25.0, 1.0, 4343)
        strain, psd, dt, _ = make_segment(w)
    elif case == "streamed16k_wait0":
        w = synth.Workload("edge22", 1 << 22, 4096.0, 30.0, 7, 2, 1.0, 6.0, False, 1, 25.0, 25.0, 1.0, 4344)
        strain, psd, dt, _ = make_segment(w)
    else:
        w = W
        strain, psd, dt, _ = make_segment(W)
    flags = CUI_PLAIN if case.startswith("plain") else 0
    thr = 0.0 if "contended" in case else 6.0
    with _bank(m=w.masses(), n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, flags=flags, snr_threshold=thr,
               ) as b:
        if case == "streamed_wait0":
            b.set_tuning(64, 16, 0, w.n_templates)
        elif case == "streamed16k_wait0":
            b.set_tuning(256, 32, 0, w.n_templates)
        b.upload(strain, psd)
        if case.startswith("streamed"):
            b.set_wait_bounds(-1, 0)
        else:
            b.set_wait_bounds(1 if "rounds1" in case else 0, -1)
        b.filter()
        with pytest.raises(CuiError) as e:
            b.peaks()
        assert e.value.status == _lib.CUI_ERR_TIMEOUT
        b.set_wait_bounds()
        b.upload(strain, psd)
        b.filter()
        peaks = b.peaks()
        trig, _ = b.triggers(allow_overflow=True) if thr == 0.0 else b.triggers()
    if thr > 0.0:
        rep = compare_bank(w, dt, psd, peaks, trig, range(w.n_templates), 0, w.n, int(w.fs), thr)
        assert rep.ok(), rep
    else:
        rep = compare_bank(w, dt, psd, peaks, trig[:0], range(w.n_templates), 0, w.n, int(w.fs), 1e9)
        assert rep.ok(), rep


def test_wait_bounds_above_the_defaults_are_rejected(seg):
    from paper_1006_4644_gb300 import CuiError, _lib

    with _bank() as b:
        for args in ((1 << 21, -1), (-1, 2 * 10 ** 9)):
            with pytest.raises(CuiError) as e:
                b.set_wait_bounds(*args)
            assert e.value.status == _lib.CUI_ERR_ARG


def test_small_segments_use_the_plain_path():
    # N < 2^12 runs the per-template path; same answers as the oracle
    w = synth.Workload("tiny", 1 << 10, 4096.0, 100.0, 4, 4, 1.0, 3.0, False, 1, 15.0, 15.0, 1.0, 99)
    strain, psd, dt, _ = make_segment(w)
    from paper_1006_4644_gb300 import Bank

    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, window=100) as b:
        b.upload(strain, psd)
        b.filter()
        p = b.peaks()
        tr, _ = b.triggers()
    rep = compare_bank(w, dt, psd, p, tr, range(w.n_templates), 0, w.n, 100, 6.0)
    assert rep.ok(), rep


def test_graph_replay_matches_direct_launches(seg):
    """cui_filter_bank replays a captured CUDA graph by default; results equal
    the directly launched kernels, across calls that change the order's
    contents (same buffer) and its length (new capture)."""
    from paper_1006_4644_gb300 import _lib

    strain, psd, _, _ = seg
    orders = [None, [5, 0, 3], [1, 2, 4], [0, 1, 2, 3, 4, 5]]
    res = {}
    for flags in (0, _lib.CUI_NO_GRAPH):
        with _bank(flags=flags, snr_threshold=4.0) as b:
            b.upload(strain, psd)
            out = []
            for o in orders:
                b.filter(order=o)
                out.append((b.peaks().copy(), b.triggers()[0]))
            res[flags] = out
    for (pa, ta), (pb, tb) in zip(res[0], res[_lib.CUI_NO_GRAPH]):
        assert np.array_equal(pa, pb)
        assert np.array_equal(ta, tb)
