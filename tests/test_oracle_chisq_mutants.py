"""The chi^2 pins catch plausible mistakes: copies of the oracle's definition
with one planted error each (equal-width instead of equal-power sub-bands, the
missing factor p, the missing z/p term, the 4 df factor dropped from the
correlators) fail the pins that the oracle passes: chi^2 ~ 0 for the exact
template and the 2p - 2 mean in Gaussian noise."""

import math

import numpy as np
import pytest

import oracle
import synth

N, FS, F_LOW = 1 << 13, 4096.0, 30.0  # df = 0.5 Hz: the 4 df factor is not 1
M1, M2, PN = 3.0, 2.0, 7


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def variant(mistake=None):
    def chisq(dtilde, psd, samples, bands):
        h, k_lo, k_hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
        df = FS / N
        k = np.arange(k_lo, k_hi)
        fac = 1.0 if mistake == "no_4df" else 4.0 * df
        terms = fac * np.asarray(dtilde)[k_lo:k_hi] * np.conj(h[k_lo:k_hi]) / psd[k_lo:k_hi]
        power = np.abs(h[k_lo:k_hi]) ** 2 / psd[k_lo:k_hi]
        pw = np.concatenate([[0.0], np.cumsum(power)])
        if mistake == "equal_width":
            edges = [len(k) * l // bands for l in range(bands + 1)]
        else:
            edges = [0] + [int(np.searchsorted(pw, pw[-1] * l / bands, side="left")) for l in range(1, bands)] + [len(k)]
        s2 = oracle.sigma2(h, psd, FS, N, k_lo, k_hi)
        out = []
        for s in samples:
            ph = np.exp(2j * np.pi * ((k * int(s)) % N) / N)
            zl = np.array([np.sum(terms[edges[l]:edges[l + 1]] * ph[edges[l]:edges[l + 1]]) for l in range(bands)])
            z = zl.sum()
            mean = 0.0 if mistake == "no_mean" else z / bands
            p = 1.0 if mistake == "no_p" else bands
            out.append(p * np.sum(np.abs(zl - mean) ** 2) / s2)
        return np.array(out)
    return chisq


def passes(chisq):
    psd = synth.psd_onesided(N, FS)
    h, lo, hi = oracle.spa_template(M1, M2, PN, F_LOW, FS, N)
    s2 = oracle.sigma2(h, psd, FS, N, lo, hi)
    d = np.zeros(N // 2 + 1, dtype=np.complex128)
    synth.add_signal(d, h, 10.0 / math.sqrt(s2), 1234, N)
    if not chisq(d, psd, [1234], 16)[0] < 1e-3 * 100.0:
        return False
    p, vals = 8, []
    for seg in range(4):
        dn = synth.noise_spectrum(11, seg, N, FS, psd, F_LOW)
        vals.append(chisq(dn, psd, range(0, N, 128), p))
    mean = np.concatenate(vals).mean()
    return abs(mean - (2 * p - 2)) < 0.1 * (2 * p - 2)


def test_unmodified_copy_and_oracle_pass():
    assert passes(variant())

    def oracle_chisq(d, psd, samples, bands):
        return oracle.chisq(d, psd, M1, M2, PN, F_LOW, FS, N, samples, bands)[0]

    assert passes(oracle_chisq)


@pytest.mark.parametrize("mistake", ["equal_width", "no_p", "no_mean", "no_4df"])
def test_planted_mistake_is_caught(mistake):
    assert not passes(variant(mistake)), mistake
