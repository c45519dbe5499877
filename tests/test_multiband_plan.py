"""Host logic of the multi-band search: the short segments' reported ranges
tile the searchable range exactly once and stay inside each segment's valid
range."""

import pytest

from paper_1006_4644_gb300.multiband import chunk_plan


@pytest.mark.parametrize("n,ns,lo,hi", [(1 << 20, 1 << 16, 40960, 61440), (1 << 12, 1 << 10, 0, 1024),
                                        (1000, 300, 50, 250), (512, 512, 10, 500), (4096, 1024, 100, 101)])
def test_chunk_plan_tiles_the_range(n, ns, lo, hi):
    plan = chunk_plan(n, ns, lo, hi)
    cover = []
    for s, a, b in plan:
        assert 0 <= s and s + ns <= n
        assert s + lo <= a < b <= s + hi
        cover.extend(range(a, b))
    assert cover == list(range(lo, n - ns + hi))


def test_chunk_plan_rejects_bad_ranges():
    with pytest.raises(ValueError):
        chunk_plan(100, 200, 0, 10)
    with pytest.raises(ValueError):
        chunk_plan(100, 50, 30, 20)
