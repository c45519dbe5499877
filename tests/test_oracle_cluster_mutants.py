"""The clustering pins catch plausible mistakes: copies of the window-maximum
definition with one planted error each (the tie on samples, the tie on
templates, the window stride, the window origin, the order of the output)
fail the hand cases or the sort-based formulation that the oracle passes."""

import numpy as np
import pytest

import oracle


def variant(mistake=None):
    def cluster(tmpl, sample, rho, lo, window):
        best = {}
        w = window + 1 if mistake == "stride" else window
        o = lo - 1 if mistake == "origin" else lo
        for i in range(len(tmpl)):
            m = (int(sample[i]) - o) // w
            ks = int(sample[i]) if mistake == "sample_tie" else -int(sample[i])
            kt = int(tmpl[i]) if mistake == "template_tie" else -int(tmpl[i])
            cand = (float(rho[i]), ks, kt)
            if m not in best or cand > best[m][0]:
                best[m] = (cand, i)
        keys = sorted(best, reverse=(mistake == "order"))
        return [best[m][1] for m in keys]
    return cluster


def passes(cluster):
    lo, W = 100, 10
    cases = [(([1, 3, 2], [101, 109, 110], [7.0, 9.0, 6.5]), [1, 2]),
             (([5, 4], [105, 103], [8.0, 8.0]), [1]),
             (([9, 2, 7], [104, 104, 104], [8.0, 8.0, 8.0]), [1]),
             (([0, 1], [119, 120], [6.1, 9.9]), [0, 1]),
             (([0, 1], [109, 110], [6.1, 9.9]), [0, 1])]
    for (t, s, r), want in cases:
        if cluster(t, s, r, lo, W) != want:
            return False
    rng = np.random.default_rng(5)
    for _ in range(20):
        n = int(rng.integers(1, 400))
        lo, W = int(rng.integers(0, 50)), int(rng.integers(1, 64))
        t = rng.integers(0, 30, n)
        s = lo + rng.integers(0, 40 * W, n)
        r = np.round(rng.uniform(6, 9, n), 1)
        win = (s - lo) // W
        order = np.lexsort((t, s, -r, win))
        first = order[np.r_[True, np.diff(win[order]) != 0]]
        if cluster(t, s, r, lo, W) != first[np.argsort(s[first], kind="stable")].tolist():
            return False
    return True


def test_unmodified_copy_and_oracle_pass():
    assert passes(variant())
    assert passes(oracle.cluster_windows)


@pytest.mark.parametrize("mistake", ["sample_tie", "template_tie", "stride", "origin", "order"])
def test_planted_mistake_is_caught(mistake):
    assert not passes(variant(mistake)), mistake
