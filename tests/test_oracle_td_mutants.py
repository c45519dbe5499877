"""The time-domain generator's pins catch plausible mistakes: the oracle's
TaylorT2 series with one planted error each (the derivative of the energy, the
sign of the series division, one energy digit, one flux term, the logarithm of
the 2.5PN phase term) must fail the stationary-phase pin that the oracle
itself passes."""

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


def spa_pin(pn_x2):
    """Psi_F2(f) = 2 pi f t(v) - 2 phi(v) - pi/4 + const along the band."""
    f = np.geomspace(20.0, 1.0 / (6 ** 1.5 * math.pi * M) * 0.99, 200)
    v = (math.pi * M * f) ** (1.0 / 3.0)
    spa_t2 = 2 * math.pi * f * td.t_of_v(v, M, ETA, pn_x2) - 2 * td.phi_of_v(v, M, ETA, pn_x2) - math.pi / 4
    diff = oracle.spa_phase(M1, M2, pn_x2, f) - spa_t2
    return np.std(diff) < 1e-9 and (pn_x2 == 5 or abs(diff.mean()) < 1e-9)


def series(num_of, sign=-1.0, e_edit=None, f_edit=None):
    """A copy of the oracle's series division with optional planted mistakes."""
    def t2(eta, pn_x2):
        e, f = td.energy_flux(eta)
        if e_edit:
            e = e_edit(list(e))
        if f_edit:
            f = f_edit(list(f))
        num = [num_of(k) * e[k] for k in range(6)]
        a = []
        for k in range(pn_x2 + 1):
            a.append(num[k] + sign * sum(a[i] * f[k - i] for i in range(k)))
        return np.array(a)
    return t2


def test_unmodified_copy_passes(monkeypatch):
    monkeypatch.setattr(td, "t2_series", series(lambda k: (k + 2) / 2.0))
    assert all(spa_pin(p) for p in (2, 3, 4, 5))


MUTANTS = {
    "energy_derivative": dict(num_of=lambda k: (k + 1) / 2.0),
    "division_sign": dict(num_of=lambda k: (k + 2) / 2.0, sign=+1.0),
    "energy_digit": dict(num_of=lambda k: (k + 2) / 2.0,
                         e_edit=lambda e: e[:2] + [e[2] * 1.001] + e[3:]),
    "flux_tail_term": dict(num_of=lambda k: (k + 2) / 2.0, f_edit=lambda f: f[:3] + [0.0] + f[4:]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_series_mistake_is_caught(monkeypatch, name):
    monkeypatch.setattr(td, "t2_series", series(**MUTANTS[name]))
    assert not all(spa_pin(p) for p in (2, 3, 4, 5)), name


def test_dropped_log_term_is_caught(monkeypatch):
    def phi_no_log(v, M_, eta, pn_x2):
        a = td.t2_series(eta, pn_x2)
        v = np.asarray(v, dtype=np.float64)
        s = sum(a[k] * (1.0 if k == 5 else v ** (k - 5) / (k - 5)) for k in range(len(a)))
        return 5.0 / (32.0 * eta) * s

    monkeypatch.setattr(td, "phi_of_v", phi_no_log)
    assert not spa_pin(5)
