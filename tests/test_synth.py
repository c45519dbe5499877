"""The seeded input generators (CPU): determinism, ranges and the published
SplitMix64 output on a known seed."""

import numpy as np

import synth


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the reference generator
    # (Steele, Lea & Flood 2014; also Vigna's splitmix64.c) are
    # 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F.
    g = synth.GAMMA
    states = np.array([1, 2, 3], dtype=np.uint64) * g
    out = synth.mix64(states)
    assert [int(x) for x in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_deterministic_and_distinct():
    a = synth.uniform(1, 2, 1000)
    b = synth.uniform(1, 2, 1000)
    c = synth.uniform(1, 3, 1000)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    # offsets address the same counter space
    assert np.array_equal(synth.uniform(1, 2, 10, 990), a[990:])
    g1, g2 = synth.normal_pairs(7, 0, 200000)
    assert abs(g1.mean()) < 0.01 and abs(g2.std() - 1) < 0.01


def test_masses_and_injections():
    m1, m2 = synth.sample_masses(3, 1, 5000, 1.0, 25.0, True)
    assert m1.min() >= 1.0 and m2.max() <= 25.0
    # log-uniform: the median of ln m sits at the midpoint
    assert abs(np.median(np.log(m1)) - np.log(25) / 2) < 0.1
    j = synth.injection_times(1, 2, 5, 0, 1 << 20, 8192)
    assert len(set(j.tolist())) == 5
    for a in j:
        for b in j:
            if a != b:
                assert min(abs(a - b), (1 << 20) - abs(a - b)) >= 8192


def test_workload_recipes():
    w = synth.WORKLOADS["seg256s_bank1024_pn35"]
    assert w.n == 1 << 20 and w.n_templates == 1024 and w.pn_x2 == 7
    t, j0, snr = w.injection_plan()
    assert len(t) == 5 and np.all((snr >= 8) & (snr <= 15))
    d = synth.WORKLOADS["seg16s_bank64_pn2"].noise()
    k0 = synth.band_start(40.0, 1 << 16, 4096.0)
    assert np.all(d[:k0] == 0) and d[-1] == 0 and np.all(d[k0:-1] != 0)
