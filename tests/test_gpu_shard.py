"""Bank sharding on the GPU: the bank split into K chirp-mass shards, each
filtered by its own Bank on this GPU (K virtual ranks run one after another),
merged, gives exactly the unsharded bank's peaks and triggers; and one rank
of ShardedSearch without a process group is the whole bank."""

import numpy as np
import pytest

import synth
from parity import make_segment

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def seg():
    from paper_1006_4644_gb300 import build

    build.build()
    w = synth.WORKLOADS["seg16s_bank64_pn2"]
    strain, psd, _, _ = make_segment(w)
    return w, strain, psd


@pytest.mark.parametrize("k", [2, 3, 5])
def test_virtual_shards_equal_the_whole_bank(seg, k):
    from paper_1006_4644_gb300 import Bank
    from paper_1006_4644_gb300.shard import merge, partition

    w, strain, psd = seg
    m1, m2 = w.masses()
    kw = dict(n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0)
    with Bank(m1, m2, **kw) as b:
        b.upload(strain, psd)
        b.filter()
        ref_peaks = b.peaks()
        ref_trig, ref_total = b.triggers()
    parts = []
    for idx in partition(m1, m2, k, n=w.n, fs=w.fs, f_low=w.f_low):
        with Bank(m1[idx], m2[idx], **kw) as b:
            b.upload(strain, psd)
            b.filter()
            parts.append((idx, b.peaks(), *b.triggers()))
    peaks, trig, total = merge(len(m1), parts)
    assert np.array_equal(peaks, ref_peaks)
    assert np.array_equal(trig, ref_trig) and total == ref_total


def test_single_rank_search_is_the_whole_bank(seg):
    from paper_1006_4644_gb300 import Bank
    from paper_1006_4644_gb300.shard import ShardedSearch

    w, strain, psd = seg
    m1, m2 = w.masses()
    ss = ShardedSearch(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0)
    peaks, trig, total = ss.search(strain, psd)
    ss.close()
    with Bank(m1, m2, n=w.n, fs=w.fs, f_low=w.f_low, pn_x2=w.pn_x2, snr_threshold=5.0) as b:
        b.upload(strain, psd)
        b.filter()
        assert np.array_equal(peaks, b.peaks())
        ref, ref_total = b.triggers()
        assert np.array_equal(trig, ref) and total == ref_total
