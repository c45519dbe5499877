"""Bank sharding (host logic): the partition, the band edges it balances on,
and a world-size-2 gloo run whose gathered result equals the single-process
one.  No GPU: the ranks filter with a host-only stand-in for Bank."""

import socket

import numpy as np
import pytest

import oracle
from paper_1006_4644_gb300.regions import chirp_mass
from paper_1006_4644_gb300.shard import band_bins, merge, partition, template_cost

import shard_worker as sw


@pytest.fixture(scope="module", autouse=True)
def _oracle():
    oracle.build()


def test_band_bins_match_the_oracle_band_edges():
    # the oracle's template support is [k_low, k_hi) (the bins with f_low <= f_k < f_ISCO, below n/2)
    rng = np.random.default_rng(3)
    for n, f_low in [(1 << 12, 30.0), (1 << 14, 20.0), (1 << 16, 40.0)]:
        for _ in range(6):
            m1, m2 = rng.uniform(1.0, 30.0, 2)
            _, lo, hi = oracle.spa_template(m1, m2, 7, f_low, 4096.0, n)
            assert band_bins([m1], [m2], n=n, fs=4096.0, f_low=f_low)[0] == max(hi - lo, 0)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_is_a_balanced_chirp_mass_split(world):
    m1, m2 = sw.bank_masses(count=501)
    kw = dict(n=1 << 16, fs=4096.0, f_low=30.0)
    shards = partition(m1, m2, world, **kw)
    assert len(shards) == world
    allidx = np.concatenate(shards)
    assert np.array_equal(np.sort(allidx), np.arange(len(m1)))  # every template exactly once
    mc = chirp_mass(m1, m2)
    for a, b in zip(shards[:-1], shards[1:]):  # contiguous chirp-mass ranges
        if len(a) and len(b):
            assert mc[a].max() <= mc[b].min()
    cost = template_cost(m1, m2, **kw)
    loads = np.array([cost[s].sum() for s in shards])
    assert loads.max() <= cost.sum() / world + cost.max() + 1e-9


def test_partition_of_fewer_templates_than_ranks():
    shards = partition([1.0, 2.0], [1.5, 3.0], 4, n=4096, fs=4096.0, f_low=30.0)
    assert sorted(np.concatenate(shards).tolist()) == [0, 1]


def test_merge_maps_shard_templates_to_bank_order():
    from paper_1006_4644_gb300 import PEAK_DTYPE, TRIGGER_DTYPE

    pk = np.zeros(2, dtype=PEAK_DTYPE)
    pk["sample"] = [10, 20]
    tr = np.zeros(2, dtype=TRIGGER_DTYPE)
    tr["tmpl"], tr["sample"] = [1, 0], [5, 7]
    peaks, trig, total = merge(4, [(np.array([3, 1]), pk, tr, 2), (np.array([0, 2]), pk, tr[:0], 0)])
    assert peaks["sample"].tolist() == [10, 20, 20, 10]
    assert trig["tmpl"].tolist() == [1, 3] and trig["sample"].tolist() == [5, 7] and total == 2


def test_two_gloo_ranks_gather_the_single_process_result(tmp_path):
    import torch.multiprocessing as mp

    from paper_1006_4644_gb300.shard import ShardedSearch

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "rank0.npz")
    mp.spawn(sw.run_rank, args=(2, port, out), nprocs=2, join=True)
    got = np.load(out)
    m1, m2 = sw.bank_masses()
    strain, psd = sw.segment()
    ref_peaks, ref_trig, ref_total = ShardedSearch(m1, m2, n=sw.N, fs=sw.FS, f_low=sw.F_LOW,
                                                   bank_factory=sw.FakeBank).search(strain, psd)
    assert np.array_equal(got["peaks"], ref_peaks)
    assert np.array_equal(got["trig"], ref_trig)
    assert int(got["total"]) == ref_total
    s0, s1 = got["shard0"], got["shard1"]
    assert len(s0) and len(s1) and len(np.intersect1d(s0, s1)) == 0


def test_library_band_rule_matches_the_oracle_and_clamps():
    """cui_template_bands (host code, no GPU) gives the oracle's template
    support [k_low, k_hi) for random masses, and clamps k_low at N/2 when
    f_low reaches Nyquist (every band empty)."""
    from paper_1006_4644_gb300 import CuiError, template_bands

    rng = np.random.default_rng(17)
    m1, m2 = rng.uniform(1.0, 60.0, 40), rng.uniform(1.0, 60.0, 40)
    for n, f_low in [(1 << 12, 30.0), (1 << 16, 10.0), (1 << 20, 20.0)]:
        k_lo, k_hi = template_bands(m1, m2, n=n, fs=4096.0, f_low=f_low)
        for t in range(len(m1)):
            _, lo, hi = oracle.spa_template(m1[t], m2[t], 7, f_low, 4096.0, n)
            if hi > lo:
                assert (k_lo, int(k_hi[t])) == (lo, hi)
            else:
                assert int(k_hi[t]) <= k_lo
    k_lo, _ = template_bands([1.4], [1.4], n=1 << 12, fs=4096.0, f_low=1e300)
    assert k_lo == 1 << 11
    with pytest.raises(CuiError):
        template_bands([1.4], [-1.0], n=1 << 12, fs=4096.0, f_low=20.0)
