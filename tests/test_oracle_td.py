"""Pins of the oracle's time-domain (TaylorT2) generator: the Newtonian closed
forms, the orbital relation dphi/dt = v^3 / M, the stationary-phase relation
to the TaylorF2 phase (itself pinned by the published energy and flux), and
the per-sample time inversion."""

import math

import numpy as np
import pytest

import oracle
from oracle import td

M1, M2 = 5.0, 3.0
M = (M1 + M2) * td.MSUN_S
ETA = M1 * M2 / (M1 + M2) ** 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_newtonian_closed_forms():
    v = np.linspace(0.05, 0.4, 50)
    assert np.allclose(td.t_of_v(v, M, ETA, 0), -5 * M / (256 * ETA * v ** 8), rtol=1e-14)
    assert np.allclose(td.phi_of_v(v, M, ETA, 0), -1.0 / (32 * ETA * v ** 5), rtol=1e-14)


@pytest.mark.parametrize("pn_x2", [0, 2, 3, 4, 5])
def test_orbital_frequency(pn_x2):
    # dphi/dt = v^3 / M along the solution, from finite differences in v
    v = np.linspace(0.08, 0.35, 40)
    h = 1e-6 * v
    dphi = td.phi_of_v(v + h, M, ETA, pn_x2) - td.phi_of_v(v - h, M, ETA, pn_x2)
    dt = td.t_of_v(v + h, M, ETA, pn_x2) - td.t_of_v(v - h, M, ETA, pn_x2)
    assert np.allclose(dphi / dt, v ** 3 / M, rtol=1e-7)


@pytest.mark.parametrize("pn_x2", [0, 2, 3, 4, 5])
def test_stationary_phase_of_t2_is_f2(pn_x2):
    # Psi_F2(f) = 2 pi f t(v) - 2 phi(v) - pi/4 + const, v = (pi M f)^(1/3)
    f = np.geomspace(20.0, 1.0 / (6 ** 1.5 * math.pi * M) * 0.99, 200)
    v = (math.pi * M * f) ** (1.0 / 3.0)
    spa_t2 = 2 * math.pi * f * td.t_of_v(v, M, ETA, pn_x2) - 2 * td.phi_of_v(v, M, ETA, pn_x2) - math.pi / 4
    diff = oracle.spa_phase(M1, M2, pn_x2, f) - spa_t2
    # a 0.1 % error in one energy or flux coefficient leaves ~1e-2 rad here
    assert np.std(diff) < 1e-9, (pn_x2, np.std(diff))
    if pn_x2 < 5:  # below 2.5PN neither phase has a free constant
        assert abs(diff.mean()) < 1e-9


def test_time_inversion_and_samples():
    fs, n, f_low = 4096.0, 1 << 15, 30.0
    hp, hx = td.td_template(M1, M2, 5, f_low, fs, n)
    on = np.nonzero(hp != 0)[0]
    assert len(on) > 1000 and on.max() == n - 1  # the chirp ends just before t = 0
    t = -(n - on) / fs
    v_lo = (math.pi * M * f_low) ** (1 / 3)
    v = td.v_of_t(t, M, ETA, 5, v_lo, 6 ** -0.5)
    assert np.allclose(td.t_of_v(v, M, ETA, 5), t, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.hypot(hp[on], hx[on]), v ** 2, rtol=1e-12)
