"""The paper's own template form on the GPU (cui_td_template): time-domain
TaylorT2 polarisations against the oracle sample for sample, and their match
with the stationary-phase bank through the filter (the mismatch of
eq:mismatch) against the oracle's match."""

import math

import numpy as np
import pytest

import oracle
import synth
from oracle import td

pytestmark = pytest.mark.gpu

N, FS, F_LOW = 1 << 16, 4096.0, 30.0
MASSES = [(5.0, 3.0), (5.0, 5.0), (10.0, 8.0), (2.0, 1.5)]


@pytest.fixture(scope="module")
def bank():
    from paper_1006_4644_gb300 import Bank, build

    build.build()
    oracle.build()
    m1 = np.array([m[0] for m in MASSES])
    m2 = np.array([m[1] for m in MASSES])
    with Bank(m1, m2, n=N, fs=FS, f_low=F_LOW, pn_x2=5, snr_threshold=1e30) as b:
        yield b


def _gpu_td(b, t, pn_x2):
    import torch

    hp = torch.empty(N, dtype=torch.float64, device="cuda")
    hx = torch.empty(N, dtype=torch.float64, device="cuda")
    b.td_template(t, hp, hx, pn_x2)
    return hp.cpu().numpy(), hx.cpu().numpy()


@pytest.mark.parametrize("pn_x2", [0, 4, 5])
def test_samples_match_the_oracle(bank, pn_x2):
    for t, (m1, m2) in enumerate(MASSES):
        hp, hx = _gpu_td(bank, t, pn_x2)
        op, ox = td.td_template(m1, m2, pn_x2, F_LOW, FS, N)
        assert np.array_equal(hp != 0, op != 0)
        scale = np.abs(op).max()
        assert np.abs(hp - op).max() <= 1e-9 * scale and np.abs(hx - ox).max() <= 1e-9 * scale, (t, pn_x2)


def test_match_with_the_spa_bank(bank):
    psd = synth.psd_onesided(N, FS)
    df = FS / N
    for t, (m1, m2) in enumerate(MASSES):
        hp, _ = _gpu_td(bank, t, 5)
        strain = hp * 1e-21  # the detector scale keeps rho^2 inside FP32
        dt = oracle.segment_spectrum(strain, FS)
        lo = int(math.ceil(F_LOW / df))
        sig_td = math.sqrt(4 * df * np.sum(np.abs(dt[lo:N // 2]) ** 2 / psd[lo:N // 2]))
        bank.upload(strain, psd)
        bank.filter()
        peak = bank.peaks()[t]
        match_gpu = peak["snr"] / sig_td
        # the oracle's match: its SPA template correlated with the same data
        h, klo, khi = oracle.spa_template(m1, m2, 5, F_LOW, FS, N)
        z = oracle.correlate(dt, h, psd, FS, N, klo, khi)
        match_or = np.abs(z).max() / math.sqrt(oracle.sigma2(h, psd, FS, N, klo, khi)) / sig_td
        assert abs(match_gpu / match_or - 1) < 1e-3, (t, match_gpu, match_or)
        assert int(peak["sample"]) in (0, N - 1, 1) or match_or < 0.9  # both coalesce at sample 0
        if m1 + m2 < 12:
            assert match_gpu > 0.98, (t, match_gpu)  # SPA and time-domain forms agree for light binaries
