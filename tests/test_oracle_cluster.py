"""Pins of the oracle's cross-template clustering (host only): hand cases for
the window edges and the tie rules, and agreement with a second, sort-based
formulation on random records."""

import numpy as np

import oracle


def test_hand_cases():
    lo, W = 100, 10
    # window 0 = [100, 110): template 3 is louder; window 1 = [110, 120): alone
    t = [1, 3, 2]
    s = [101, 109, 110]
    r = [7.0, 9.0, 6.5]
    assert oracle.cluster_windows(t, s, r, lo, W) == [1, 2]
    # equal rho: the lower sample wins, whatever the template
    assert oracle.cluster_windows([5, 4], [105, 103], [8.0, 8.0], lo, W) == [1]
    # equal rho and sample: the lower template wins
    assert oracle.cluster_windows([9, 2, 7], [104, 104, 104], [8.0, 8.0, 8.0], lo, W) == [1]
    # the last sample of a window and the first of the next never merge
    assert oracle.cluster_windows([0, 1], [119, 120], [6.1, 9.9], lo, W) == [0, 1]
    assert oracle.cluster_windows([], [], [], lo, W) == []


def test_agrees_with_a_sort_based_formulation():
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(1, 400))
        lo, W = int(rng.integers(0, 50)), int(rng.integers(1, 64))
        t = rng.integers(0, 30, n)
        s = lo + rng.integers(0, 40 * W, n)
        r = np.round(rng.uniform(6, 9, n), 1)  # coarse values make ties common
        got = oracle.cluster_windows(t, s, r, lo, W)
        # sort by (window, -rho, sample, template); the first record of each window wins
        win = (s - lo) // W
        order = np.lexsort((t, s, -r, win))
        first = order[np.r_[True, np.diff(win[order]) != 0]]
        want = first[np.argsort(s[first], kind="stable")]
        assert got == want.tolist()
