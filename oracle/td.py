"""Time-domain inspiral templates -- TEST INFRASTRUCTURE ONLY (same rules as the
rest of ``oracle``: only tests, the smoke check and the benchmark's CPU leg
use it; the library never imports it).

The paper's own generator (Sec. "template generation"): the two polarisations
of a circular inspiral in the time domain, post-Newtonian order 2.5 in phase
and 0 in amplitude, later Fourier transformed and normalised.  The paper
prints no formula; the orbital evolution here is the TaylorT2 form of the PN
literature it cites, derived from the binding energy and the energy flux of
circular orbits (v = (M omega)^(1/3), x = v^2):

    E(v) = -(1/2) eta M v^2 [1 + e1 v^2 + e2 v^4]
    F(v) = (32/5) eta^2 v^10 [1 + f2 v^2 + f3 v^3 + f4 v^4 + f5 v^5]

    dt/dv   = -E'(v) / F(v) = (5 M / (32 eta)) v^-9 sum_k a_k v^k
    dphi/dv = (v^3 / M) dt/dv

with the series a_k from dividing the two brackets (kept to v^pn_x2) and
both relations integrated term by term (t_c = phi_c = 0; the v^5 term of the
phase integrates to a logarithm).  phi is the orbital phase; the waves are
h_+ = v^2 cos 2 phi and h_x = v^2 sin 2 phi (Newtonian amplitude, up to a
constant), between f_low and the innermost stable orbit v = 6^(-1/2).
"""

from __future__ import annotations

import math

import numpy as np

MSUN_S = 4.925490947e-6  # G M_sun / c^3 (s)


def energy_flux(eta: float):
    """Bracket coefficients (powers v^0 .. v^5) of E and F to the orders the
    2.5PN phase needs."""
    pi = math.pi
    e = [1.0, 0.0, -0.75 - eta / 12.0, 0.0, -27.0 / 8.0 + 19.0 * eta / 8.0 - eta * eta / 24.0, 0.0]
    f = [1.0, 0.0, -1247.0 / 336.0 - 35.0 * eta / 12.0, 4.0 * pi,
         -44711.0 / 9072.0 + 9271.0 * eta / 504.0 + 65.0 * eta * eta / 18.0,
         -(8191.0 / 672.0 + 583.0 * eta / 24.0) * pi]
    return e, f


def t2_series(eta: float, pn_x2: int):
    """a_0 .. a_pn_x2 of dt/dv = (5 M / (32 eta)) v^-9 sum_k a_k v^k."""
    if not 0 <= pn_x2 <= 5:
        raise ValueError("the time-domain generator keeps up to 2.5PN (pn_x2 <= 5)")
    e, f = energy_flux(eta)
    # -E'(v) / (eta M v) = 1 + 2 e1 v^2 + 3 e2 v^4: the derivative of v^2 [sum e_k v^k] / 2
    num = [(k + 2) / 2.0 * e[k] for k in range(6)]
    a = []
    for k in range(pn_x2 + 1):  # series division num / f
        a.append(num[k] - sum(a[i] * f[k - i] for i in range(k)))
    return np.array(a)


def t_of_v(v, M: float, eta: float, pn_x2: int):
    a = t2_series(eta, pn_x2)
    v = np.asarray(v, dtype=np.float64)
    s = sum(a[k] * v ** (k - 8) / (k - 8) for k in range(len(a)))
    return 5.0 * M / (32.0 * eta) * s


def dt_dv(v, M: float, eta: float, pn_x2: int):
    a = t2_series(eta, pn_x2)
    v = np.asarray(v, dtype=np.float64)
    return 5.0 * M / (32.0 * eta) * sum(a[k] * v ** (k - 9) for k in range(len(a)))


def phi_of_v(v, M: float, eta: float, pn_x2: int):
    a = t2_series(eta, pn_x2)
    v = np.asarray(v, dtype=np.float64)
    s = sum(a[k] * (np.log(v) if k == 5 else v ** (k - 5) / (k - 5)) for k in range(len(a)))
    return 5.0 / (32.0 * eta) * s


def v_of_t(t, M: float, eta: float, pn_x2: int, v_lo: float, v_hi: float):
    """Solve t(v) = t by Newton from the Newtonian inverse (t < 0), clamped to
    [v_lo, v_hi]."""
    t = np.asarray(t, dtype=np.float64)
    v = np.clip((5.0 * M / (256.0 * eta * np.maximum(-t, 1e-300))) ** 0.125, v_lo, v_hi)
    for _ in range(30):
        dv = (t_of_v(v, M, eta, pn_x2) - t) / dt_dv(v, M, eta, pn_x2)
        v = np.clip(v - dv, v_lo, v_hi)
        if np.all(np.abs(dv) <= 1e-15 * v):
            break
    return v


def td_template(m1: float, m2: float, pn_x2: int, f_low: float, fs: float, n: int):
    """(h_+, h_x): n samples, sample j at t_j = -((n - j) mod n) / fs, so the
    chirp ends (coalesces) at t = 0 = sample 0 and runs backwards through the
    end of the buffer; zero outside [t(v_low), t(v_isco)] and for t < -n/fs."""
    M = (m1 + m2) * MSUN_S
    eta = m1 * m2 / (m1 + m2) ** 2
    v_lo = (math.pi * M * f_low) ** (1.0 / 3.0)
    v_hi = 1.0 / math.sqrt(6.0)
    j = np.arange(n)
    t = -((n - j) % n) / fs
    t_lo, t_hi = float(t_of_v(v_lo, M, eta, pn_x2)), float(t_of_v(v_hi, M, eta, pn_x2))
    on = (t >= t_lo) & (t <= t_hi) & (j != 0)
    v = v_of_t(t[on], M, eta, pn_x2, v_lo, v_hi)
    ph = 2.0 * phi_of_v(v, M, eta, pn_x2)
    hp, hx = np.zeros(n), np.zeros(n)
    hp[on] = v * v * np.cos(ph)
    hx[on] = v * v * np.sin(ph)
    return hp, hx
