"""Pins of the oracle's stationary-phase template (CPU).

The paper prints no template formula (Sec. "template generation" only names
the PN orders), so the template is pinned to physics fixed elsewhere:
* amplitude f^(-7/6) and the band [f_low, f_ISCO) with f_ISCO from SI
  constants (IAU nominal solar mass parameter), not the oracle's constant;
* the Newtonian chirp time tau_0(f) in closed form (stationary phase:
  dPsi/df = 2 pi t(f));
* every PN coefficient, through d^2Psi/df^2 = 2 pi dt/df with dt/dv =
  -(dE/dv)/F built from the published binding energy and flux
  (tests/golden/pn_energy_flux.json) by truncated power-series arithmetic;
* the time-domain support of the template (the chirp ends at t = 0, i.e. at
  the end of the circular buffer), which fixes the sign convention.
"""

import json
import math
import os

import numpy as np
import pytest
import sympy as sp

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pn_energy_flux.json")
# IAU 2015 Resolution B3 nominal solar mass parameter and the SI speed of light
GM_SUN = 1.3271244e20
C_LIGHT = 299792458.0
MSUN_S = GM_SUN / C_LIGHT**3


@pytest.mark.parametrize("f_low", [40.0, 33.3])  # f_low / df integer and not
def test_amplitude_and_band(f_low):
    n, fs = 1 << 16, 4096.0
    for m1, m2 in [(1.0, 1.0), (1.7, 2.9), (10.0, 10.0), (3.0, 1.2)]:
        h, k_lo, k_hi = oracle.spa_template(m1, m2, 4, f_low, fs, n)
        df = fs / n
        f_isco = 1.0 / (6.0**1.5 * math.pi * (m1 + m2) * MSUN_S)
        assert k_lo == math.ceil(f_low / df)
        assert k_hi == min(math.ceil(f_isco / df), n // 2)
        k = np.arange(n // 2 + 1)
        band = (k >= k_lo) & (k < k_hi)
        assert np.all(h[~band] == 0)
        a = np.abs(h[band]) * (k[band] * df) ** (7.0 / 6.0)
        assert np.max(np.abs(a - 1.0)) < 1e-13


def test_band_empty_for_heavy_templates():
    # f_ISCO below f_low: the template has no bins at all
    h, k_lo, k_hi = oracle.spa_template(60.0, 60.0, 7, 40.0, 4096.0, 1 << 12)
    assert k_hi <= k_lo and np.all(h == 0)


def _d2(P, f):
    h = f * 2e-3
    return (-P(f + 2 * h) + 16 * P(f + h) - 30 * P(f) + 16 * P(f - h) - P(f - 2 * h)) / (12 * h * h)


def _d1(P, f):
    h = f * 1e-3
    return (-P(f + 2 * h) + 8 * P(f + h) - 8 * P(f - h) + P(f - 2 * h)) / (12 * h)


@pytest.mark.parametrize("m1,m2", [(1.0, 1.0), (1.4, 1.4), (3.0, 10.0), (20.0, 20.0)])
def test_newtonian_chirp_time(m1, m2):
    # t(f) = -tau_0(f), tau_0 = 5 / (256 pi f eta) (pi M f)^(-5/3)
    M = (m1 + m2) * MSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    f = np.array([20.0, 40.0, 80.0, 150.0])
    f = f[f < 1.0 / (6.0**1.5 * math.pi * M)]
    tau0 = 5.0 / (256.0 * math.pi * f * eta) * (math.pi * M * f) ** (-5.0 / 3.0)
    got = _d1(lambda x: oracle.spa_phase(m1, m2, 0, x), f) / (2 * math.pi)
    assert np.max(np.abs(got / -tau0 - 1.0)) < 1e-7


def _energy_flux():
    g = json.load(open(GOLDEN))
    eta = sp.Symbol("eta")
    ns = {"eta": eta, "pi": sp.pi, "EulerGamma": sp.EulerGamma}
    fns = {}
    for grp in ("energy", "flux"):
        for k, s in g[grp].items():
            if k != "form":
                fns[k] = sp.lambdify(eta, sp.sympify(s, locals=ns), "math")
    return fns


def _series_inv(b, n):
    c = [0.0] * n
    c[0] = 1.0 / b[0]
    for k in range(1, n):
        c[k] = -sum(b[i] * c[k - i] for i in range(1, k + 1)) / b[0]
    return c


def _series_mul(a, b, n):
    return [sum(a[i] * b[k - i] for i in range(k + 1)) for k in range(n)]


def _psi2_from_energy_flux(fns, m1, m2, pn_x2, f):
    """2 pi dt/df with dt/dv = -(dE/dv)/F, the ratio expanded in v and
    truncated after v^pn_x2 (the consistent TaylorF2 truncation)."""
    M = (m1 + m2) * MSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    out = []
    for ff in f:
        v = (math.pi * M * ff) ** (1.0 / 3.0)
        e1, e2, e3 = fns["e1"](eta), fns["e2"](eta), fns["e3"](eta)
        # d/dv [v^2 (1 + e1 v^2 + e2 v^4 + e3 v^6)] / (2 v)
        num = [1.0, 0.0, 2 * e1, 0.0, 3 * e2, 0.0, 4 * e3, 0.0]
        den = [1.0, 0.0, fns["f2"](eta), fns["f3"](eta), fns["f4"](eta), fns["f5"](eta),
               fns["f6"](eta) + fns["f6l"](eta) * (math.log(16.0) + 2.0 * math.log(v)), fns["f7"](eta)]
        s = _series_mul(num, _series_inv(den, 8), 8)
        S = sum(s[k] * v**k for k in range(pn_x2 + 1))
        dt_dv = 5.0 * M / (64.0 * eta) * 2.0 * v**-9 * S
        dv_df = math.pi * M / (3.0 * v * v)
        out.append(2.0 * math.pi * dt_dv * dv_df)
    return np.array(out)


@pytest.mark.parametrize("m1,m2", [(1.0, 1.0), (1.4, 1.4), (1.0, 10.0), (5.0, 25.0), (12.0, 30.0)])
@pytest.mark.parametrize("pn_x2", [0, 2, 3, 4, 5, 6, 7])
def test_pn_phase_against_energy_and_flux(m1, m2, pn_x2):
    fns = _energy_flux()
    M = (m1 + m2) * MSUN_S
    f = np.array([20.0, 45.0, 90.0, 200.0, 400.0, 900.0])
    f = f[f < 0.95 / (6.0**1.5 * math.pi * M)]
    got = _d2(lambda x: oracle.spa_phase(m1, m2, pn_x2, x), f)
    want = _psi2_from_energy_flux(fns, m1, m2, pn_x2, f)
    assert np.max(np.abs(got / want - 1.0)) < 5e-8


def test_pn_orders_are_distinguished():
    # the test above is sensitive to each order: dropping the top term of a
    # 3.5PN phase moves d^2Psi/df^2 far beyond its tolerance
    fns = _energy_flux()
    f = np.array([100.0, 200.0])
    a = _psi2_from_energy_flux(fns, 1.4, 1.4, 7, f)
    b = _psi2_from_energy_flux(fns, 1.4, 1.4, 6, f)
    assert np.min(np.abs(a / b - 1.0)) > 1e-5


def test_time_domain_support_ends_at_coalescence():
    # 10+10 Msun, f_low 40 Hz, N = 65536 at 4096 Hz, Newtonian phase:
    # the template's energy sits in the last ~tau_0(f_low) before t = 0,
    # which is the end of the circular buffer.
    n, fs, f_low, m = 1 << 16, 4096.0, 40.0, 10.0
    h, k_lo, k_hi = oracle.spa_template(m, m, 0, f_low, fs, n)
    full = np.zeros(n, complex)
    full[: n // 2 + 1] = h
    full[n // 2 + 1 :] = np.conj(h[1 : n // 2][::-1])
    ht = oracle.fft(full, +1).real
    e = ht**2
    M = 2 * m * MSUN_S
    tau0 = 5.0 / (256.0 * math.pi * f_low * 0.25) * (math.pi * M * f_low) ** (-5.0 / 3.0)
    span = int(1.1 * tau0 * fs)
    ring = int(0.05 * fs)  # the sharp cut at f_ISCO rings for a few ms around t = 0
    assert e[n - span :].sum() + e[:ring].sum() >= 0.99 * e.sum()
    # with the opposite sign convention the chirp would fill [0, tau_0) instead
    assert e[ring : n // 2].sum() <= 0.01 * e.sum()
