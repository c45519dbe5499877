"""Pins of the prescreen oracle's optimiser step, feature standardisation and
ensemble scores (CPU).  Adam (Kingma and Ba 2015, Algorithm 1) is pinned by
cases whose result follows by hand: a constant gradient, whose bias-corrected
moments equal g and g^2 exactly, so every step moves theta by
lr g / (|g| + eps); two steps of opposite gradients worked out by hand; a tiny
gradient that fixes where eps sits; a zero gradient that only decays the
moments.  Copies of the step with one planted mistake each (no bias
correction, eps inside the root, the two decay rates swapped, the sign of the
update, the second moment accumulated without its decay) fail a pin that the
oracle passes."""

import math

import numpy as np
import pytest

from oracle import prescreen as ps


def variant(mistake=None):
    def step(theta, m, v, g, t, lr, b1, b2, eps):
        theta, m, v, g = (np.asarray(a, dtype=np.float64) for a in (theta, m, v, g))
        if mistake == "swap":
            b1, b2 = b2, b1
        m_t = b1 * m + (1 - b1) * g
        v_t = (v + g * g) if mistake == "v_sum" else b2 * v + (1 - b2) * g * g
        mh = m_t if mistake == "no_bias" else m_t / (1 - b1 ** t)
        vh = v_t if mistake == "no_bias" else v_t / (1 - b2 ** t)
        den = np.sqrt(vh + eps) if mistake == "eps_inside" else np.sqrt(vh) + eps
        upd = lr * mh / den
        return (theta + upd if mistake == "sign" else theta - upd), m_t, v_t
    return step


def passes(step):
    ok = True
    # constant gradient: three steps of exactly lr g / (|g| + eps) each
    th, m, v = np.array([0.5, -2.0]), np.zeros(2), np.zeros(2)
    g = np.array([0.2, -3.0])
    for t in (1, 2, 3):
        th, m, v = step(th, m, v, g, t, 0.01, 0.9, 0.999, 1e-8)
    ok &= np.allclose(th, [0.5 - 0.03 * 0.2 / (0.2 + 1e-8), -2.0 + 0.03 * 3.0 / (3.0 + 1e-8)], rtol=0, atol=1e-15)
    # g1 = 1, g2 = -1, eps = 0, lr = 0.1: theta1 = -0.1; the corrected moments
    # of step 2 are (0.9 - 1) / 1.9 and (0.999 + 1) / 1.999 = 1, so
    # theta2 = -0.1 + 0.1 * 0.1 / 1.9 = -0.09473684210526316
    th, m, v = step(np.zeros(1), np.zeros(1), np.zeros(1), np.ones(1), 1, 0.1, 0.9, 0.999, 0.0)
    ok &= abs(th[0] + 0.1) < 1e-15
    th, m, v = step(th, m, v, -np.ones(1), 2, 0.1, 0.9, 0.999, 0.0)
    ok &= abs(th[0] + 0.09473684210526316) < 1e-15
    ok &= abs(m[0] - (0.9 * 0.1 - 0.1)) < 1e-15 and abs(v[0] - (0.999 * 0.001 + 0.001)) < 1e-15
    # g = 1e-9, eps = 1e-8: the first step is lr * 1e-9 / (1e-9 + 1e-8) = lr / 11
    th, _, _ = step(np.zeros(1), np.zeros(1), np.zeros(1), np.full(1, 1e-9), 1, 0.011, 0.9, 0.999, 1e-8)
    ok &= abs(th[0] + 0.001) < 1e-15
    # zero gradient: the moments decay by exactly b1 and b2
    th, m, v = step(np.ones(1), np.full(1, 0.5), np.full(1, 0.25), np.zeros(1), 7, 0.1, 0.9, 0.999, 1e-8)
    ok &= abs(m[0] - 0.45) < 1e-15 and abs(v[0] - 0.24975) < 1e-15
    return bool(ok)


def test_oracle_adam_passes_the_hand_cases():
    assert passes(variant())
    assert passes(ps.adam_step)


@pytest.mark.parametrize("mistake", ["no_bias", "eps_inside", "swap", "sign", "v_sum"])
def test_planted_adam_mistake_is_caught(mistake):
    assert not passes(variant(mistake)), mistake


def test_fit_norm_closed_forms():
    # band 0 constant 3 (zero spread reads 1), band 1 -1/+1 equally often,
    # band 2 the values 0, 2, 4 equally often: mean 2, std sqrt(8/3)
    f = np.zeros((3, 3, 4))
    f[:, 0, :] = 3.0
    f[:, 1, :] = np.array([-1.0, 1.0, -1.0, 1.0])
    f[0, 2, :], f[1, 2, :], f[2, 2, :] = 0.0, 2.0, 4.0
    mean, sd = ps.fit_norm(f)
    assert np.allclose(mean, [3.0, 0.0, 2.0], atol=1e-15)
    assert np.allclose(sd, [1.0, 1.0, math.sqrt(8.0 / 3.0)], atol=1e-15)
    z = ps.standardise(f[2], mean, sd)
    assert np.allclose(z[2], 2.0 / math.sqrt(8.0 / 3.0)) and np.allclose(z[0], 0.0) and np.allclose(z[1], f[2, 1])


def test_ensemble_probabilities_by_hand():
    # softmax([0, ln 3]) = [1/4, 3/4] and softmax([ln 3, 0]) = [3/4, 1/4]: mean [1/2, 1/2]
    p = ps.ensemble_probabilities([[0.0, math.log(3.0)], [math.log(3.0), 0.0]])
    assert np.allclose(p, [0.5, 0.5], atol=1e-15)
    z = np.array([0.3, -1.2, 2.0, 0.0])
    assert np.allclose(ps.ensemble_probabilities([z]), np.exp(z) / np.exp(z).sum(), atol=1e-15)
    assert np.allclose(ps.ensemble_probabilities([z, z + 5.0, z]), np.exp(z) / np.exp(z).sum(), atol=1e-15)
