"""The stored oracle filter-output labels of the prescreen
(tests/prescreen_labels/oracle_response_seed4.npz, written by
make_oracle_labels.py there from oracle/ and synth/ only) are what the oracle
gives: a few regions of a few segments are recomputed here, template by
template, with the same trigger rule (CPU).  Also the file's shape and the
physics it must show: no region responds far above the injected SNR, and
loud injections make some region respond at rho >= 8."""

import os

import numpy as np
import pytest

import oracle
import synth
from oracle import prescreen as ops
from prescreen_data import make_segments

HERE = os.path.dirname(os.path.abspath(__file__))
PATH = os.path.join(HERE, "prescreen_labels", "oracle_response_seed4.npz")


@pytest.fixture(scope="module")
def labels():
    if not os.path.exists(PATH):
        pytest.skip("no stored labels")
    return np.load(PATH)


def test_shape_and_physics(labels):
    r, snr = labels["response"], labels["snr"]
    assert r.shape == (len(snr), 100) and len(snr) >= 256
    assert np.all(r >= 0) and np.all(r.max(axis=1) <= snr + 5.0)
    loud = snr >= 14.0
    assert np.mean(r[loud].max(axis=1) >= 8.0) > 0.9


@pytest.mark.parametrize("seg", [0, 7])
def test_regions_recomputed_by_the_oracle(labels, seg):
    import sys

    sys.path.insert(0, os.path.join(HERE, "prescreen_labels"))
    from make_oracle_labels import F_LOW, FS, N, REGIONS, SEED, WINDOW, region_response

    oracle.build()
    psd = synth.psd_onesided(N, FS)
    bankw = synth.WORKLOADS["seg256s_bank10k_pn35"]
    m1, m2 = bankw.masses()
    groups, bounds = ops.regions_of_bank(m1, m2, REGIONS)
    stored = labels["response"][seg].astype(np.float64)
    # the strongest region, one silent region and one in between
    order = np.argsort(-stored, kind="stable")
    pick = sorted({int(order[0]), int(order[len(order) // 2]), int(order[-1])})
    d, _, meta = make_segments(SEED, int(labels["start"]) + seg, 1, N, FS, F_LOW, psd, bounds, REGIONS)
    assert meta[0]["j0"] == labels["j0"][seg]
    dt = oracle.segment_spectrum(synth.strain_from_spectrum(d[0], N, FS), FS)
    tm = np.concatenate([groups[r] for r in pick])
    res = oracle.filter_bank(dt, psd, m1[tm], m2[tm], 7, F_LOW, FS, N, window=WINDOW, thr=6.0)
    region_of = np.empty(len(m1), dtype=np.int64)
    for r, g in enumerate(groups):
        region_of[g] = r
    got = region_response([(x["trig_j"], x["trig_rho"]) for x in res], region_of[tm], meta[0]["j0"])
    for r in pick:
        assert np.float32(got[r]) == np.float32(stored[r]), (seg, r, got[r], stored[r])
