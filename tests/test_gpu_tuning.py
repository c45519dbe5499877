"""Every tiling the autotuner can choose gives the oracle's answers (GPU), and
the autotuner leaves a valid, timed tiling selected."""

import itertools

import numpy as np
import pytest

import synth
from parity import compare_bank, make_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()


def _tilings(bank, n):
    from paper_1006_4644_gb300 import CuiError

    out = []
    for n1, cc, rpc in itertools.product([64, 128, 256], [16, 32, 64], [0, 1, 2, 4, 8, 16, 32]):
        try:
            bank.set_tuning(n1, cc, rpc, 3)
            out.append((n1, cc, rpc))
        except CuiError:
            pass
    return out


@pytest.mark.parametrize("log2n", [14, 20])
def test_every_tiling_matches_the_oracle(log2n):
    from paper_1006_4644_gb300 import Bank

    n = 1 << log2n
    w = synth.Workload(f"tile{log2n}", n, 4096.0, 30.0, 7, 7, 1.0, 8.0, False, 1, 15.0, 15.0, 1.0, 505 + log2n)
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0) as b:
        b.upload(strain, psd)
        tilings = _tilings(b, n)
        assert len(tilings) >= (2 if log2n == 14 else 4), tilings
        for n1, cc, rpc in tilings:
            b.set_tuning(n1, cc, rpc, 3)  # batches of 3 leave a ragged last batch
            assert b.tuning() == {"n1": n1, "ccols": cc, "rpc": rpc, "batch": 3}
            b.filter()
            peaks = b.peaks()
            trig, _ = b.triggers()
            rep = compare_bank(w, dt, psd, peaks, trig, range(w.n_templates), 0, n, int(w.fs), 5.0)
            assert rep.ok(), (n1, cc, rpc, rep)


@pytest.mark.parametrize("n1,cc", list(itertools.product([64, 128, 256], [16, 32, 64])))
def test_full_template_groups_match_the_oracle(n1, cc):
    """Batches that fill every pass-1 CTA with its full group of templates, at
    the smallest CTAs (n1 = 64 with 16 columns is 64 threads)."""
    from paper_1006_4644_gb300 import Bank, CuiError

    n = 1 << 14
    w = synth.Workload("tile14g", n, 4096.0, 30.0, 7, 40, 1.0, 8.0, False, 1, 15.0, 15.0, 1.0, 521)
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0) as b:
        b.upload(strain, psd)
        for rpc in (0, 1, 2, 4, 8, 16, 32):
            try:
                b.set_tuning(n1, cc, rpc, w.n_templates)
                break
            except CuiError:
                continue
        else:
            pytest.skip("no pass-2 tiling for this n1")
        b.filter()
        peaks = b.peaks()
        trig, _ = b.triggers()
    rep = compare_bank(w, dt, psd, peaks, trig, range(w.n_templates), 0, n, int(w.fs), 5.0)
    assert rep.ok(), (n1, cc, rep)


def test_autotune_selects_a_valid_tiling():
    from paper_1006_4644_gb300 import Bank, CuiError

    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, _, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2) as b:
        with pytest.raises(CuiError):
            b.autotune()  # needs a segment
        b.upload(strain, psd)
        b.filter()
        ref = b.peaks()
        tu, ms = b.autotune(reps=1)
        assert ms > 0 and b.tuning() == tu
        b.filter()
        p = b.peaks()
    assert np.array_equal(p["sample"], ref["sample"])
    assert np.max(np.abs(p["snr"] - ref["snr"]) / ref["snr"]) < 1e-5


@pytest.mark.parametrize("log2n,n1,count,batch", [(18, 64, 5, 5), (19, 128, 3, 2), (20, 256, 1, 1),
                                                  (20, 256, 3, 3), (20, 256, 7, 4), (22, 256, 1, 1),
                                                  (22, 256, 3, 2)])
def test_streamed_pass2_equals_row_pair_kernel(log2n, n1, count, batch):
    """The streamed persistent pass 2 (rpc 0: rows copied into shared memory
    by the bulk-copy engine) against the one-row-per-CTA kernels.  Row pairs
    of 4096 points on two teams per CTA run the same arithmetic in the same
    order, so peaks and triggers are bit-identical.  The 16384-point rows of
    2^22 are split four ways in frequency and transformed as two packed
    4096-point transforms, a different order of the same sums: peaks agree to
    FP32 rounding and both kernels match the FP64 oracle.  The cases cover
    fewer row pairs than SMs (one template at 2^20: 128 row pairs, the second
    team idle), both teams, CTAs with one and with two rows at 2^22, ragged
    last batches, and a valid range that cuts rows; the error word must stay
    clear (a bounded bulk-copy wait that gave up would read CUI_ERR_TIMEOUT)."""
    from paper_1006_4644_gb300 import Bank

    n = 1 << log2n
    w = synth.Workload(f"stream{log2n}", n, 4096.0, 30.0, 7, count, 1.0, 8.0, False, 1, 15.0, 15.0, 1.0,
                       611 + log2n + count)
    strain, psd, dt, _ = make_segment(w)
    m1, m2 = w.masses()
    lo, hi = n // 7, n - n // 9
    out = {}
    for rpc in (1, 0):
        with Bank(m1, m2, n=n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=4.5, window=1000,
                  valid=(lo, hi)) as b:
            b.upload(strain, psd)
            b.set_tuning(n1, 32 if log2n == 22 else 16, rpc, batch)
            b.filter()
            b.filter()  # a second call over the same buffers
            out[rpc] = (b.peaks(), b.triggers()[0])
    if log2n < 22:
        assert np.array_equal(out[0][0], out[1][0])
        assert np.array_equal(out[0][1], out[1][1])
    else:
        a, b = out[0][0], out[1][0]
        assert np.max(np.abs(a["snr"] - b["snr"]) / b["snr"]) < 2e-6
        assert np.max(np.abs(np.angle(np.exp(1j * (a["phase"] - b["phase"]))))) < 2e-5
        rep1 = compare_bank(w, dt, psd, out[1][0], out[1][1], range(w.n_templates), lo, hi, 1000, 4.5)
        assert rep1.ok(), rep1
    rep = compare_bank(w, dt, psd, out[0][0], out[0][1], range(w.n_templates), lo, hi, 1000, 4.5)
    assert rep.ok(), rep
