"""cui_results returns exactly what cui_peaks and cui_triggers return, both
when the trigger records fit the staged prefix and when a count larger than
the previous call's needs the second copy (GPU)."""

import numpy as np
import pytest

import synth
from parity import make_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1006_4644_gb300 import build

    build.build()


@pytest.mark.parametrize("thr,window", [(6.0, 256), (3.0, 64)])
def test_results_equal_separate_read_outs(thr, window):
    from paper_1006_4644_gb300 import Bank

    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, _, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=thr, window=window) as b:
        b.upload(strain, psd)
        for _ in range(2):  # the second call reads with the first call's count as its hint
            b.filter()
            peaks, trig, total = b.results()
            assert np.array_equal(peaks, b.peaks())
            t2, total2 = b.triggers()
            assert total == total2 and np.array_equal(trig, t2)
    if thr < 4:
        assert total > 2048  # more than the first call's staged prefix


def test_results_overflow_and_errors():
    from paper_1006_4644_gb300 import Bank, CuiError

    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, _, _ = make_segment(w)
    m1, m2 = w.masses()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=3.5, window=256) as b:
        b.upload(strain, psd)
        with pytest.raises(CuiError):  # no filter call yet
            b.results()
        b.filter()
        peaks, trig, total = b.results(capacity=10, allow_overflow=True)
        assert len(trig) == 10 and total > 10
        with pytest.raises(CuiError):
            b.results(capacity=10)
