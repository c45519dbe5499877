"""Region ranking (cui_prescreen_rank, host code in the library, no GPU):
the template order equals the plain formulation (the oracle's chirp mass, a
stable sort, numpy's equal-count split into regions, and a stable descending
sort of the scores) index for index, including ties in mass and in score,
fewer templates than regions, top_k of 0 and above the region count; bad
arguments are errors."""

import numpy as np
import pytest

from oracle import prescreen as ops


def plain_order(m1, m2, scores, top_k):
    # the oracle's regions, written out so that empty groups (fewer templates
    # than regions) are allowed
    groups = np.array_split(np.argsort(ops.chirp_mass(m1, m2), kind="stable"), len(scores))
    ranked = np.argsort(-np.asarray(scores, dtype=np.float32), kind="stable")[:top_k]
    parts = [groups[r] for r in ranked]
    return np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, dtype=np.int32)


@pytest.fixture(scope="module")
def rank():
    from paper_1006_4644_gb300 import build, prescreen_rank

    build.build()
    return prescreen_rank


def test_random_banks(rank):
    rng = np.random.default_rng(11)
    for _ in range(40):
        n = int(rng.integers(0, 3000))
        regions = int(rng.integers(1, 257))
        m1 = rng.uniform(1.0, 50.0, n)
        m2 = rng.uniform(1.0, 50.0, n)
        if n > 4:  # exact repeats of bank points: equal chirp mass, bank order decides
            m1[: n // 4] = m1[n // 4: 2 * (n // 4)]
            m2[: n // 4] = m2[n // 4: 2 * (n // 4)]
        scores = rng.normal(size=regions).astype(np.float32)
        if regions > 3:  # equal scores: the lower region first
            scores[1::3] = scores[0]
        top_k = int(rng.integers(0, regions + 5))
        want = plain_order(m1, m2, scores, top_k)
        got = rank(m1, m2, scores, top_k)
        assert got.dtype == np.int32 and np.array_equal(got, want), (n, regions, top_k)


def test_default_is_the_whole_bank_once(rank):
    rng = np.random.default_rng(3)
    m1, m2 = rng.uniform(1, 10, 1000), rng.uniform(1, 10, 1000)
    got = rank(m1, m2, rng.normal(size=100))
    assert np.array_equal(np.sort(got), np.arange(1000))


def test_errors(rank):
    from paper_1006_4644_gb300 import CuiError

    m = np.ones(4)
    with pytest.raises(CuiError):
        rank(m, np.array([1.0, 1.0, 0.0, 1.0]), np.zeros(2))
    with pytest.raises(CuiError):
        rank(m, m, np.array([0.0, np.nan]))
    with pytest.raises(CuiError):
        rank(m, m, np.zeros(0))
    with pytest.raises(CuiError):
        rank(m, m, np.zeros(2), top_k=-1)


def test_region_plan_matches_the_plain_formulation():
    """cui_regions_create / cui_regions_order (the bank sorted once, reused for
    many score vectors) give the same orders as the plain formulation."""
    from paper_1006_4644_gb300 import Regions, build

    build.build()
    rng = np.random.default_rng(29)
    for n, regions in [(0, 5), (7, 10), (1000, 100), (10_000, 100), (2999, 256)]:
        m1, m2 = rng.uniform(1.0, 50.0, n), rng.uniform(1.0, 50.0, n)
        with Regions(m1, m2, regions) as plan:
            for _ in range(5):
                scores = rng.normal(size=regions).astype(np.float32)
                scores[::4] = scores[0]
                top_k = int(rng.integers(0, regions + 3))
                assert np.array_equal(plan.order(scores, top_k), plain_order(m1, m2, scores, top_k))
