"""Pins of the oracle's transforms (CPU): the textbook radix-2 FFT against the
naive DFT, the naive DFT against numpy's FFT (an independent library), closed
forms and Parseval.  The data spectrum (X(f) of eq:matchedfilter) is checked
against numpy's real FFT."""

import numpy as np
import pytest

import oracle


def _rand(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 64, 256, 1024, 4096])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_naive_dft(n, sign):
    x = _rand(n, n + sign)
    a = oracle.fft(x, sign)
    b = oracle.dft(x, sign)
    assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("n", [8, 60, 512, 1000])
def test_naive_dft_matches_numpy(n):
    # the naive DFT has no power-of-two restriction; numpy fixes the sign
    x = _rand(n, 7 * n)
    assert np.allclose(oracle.dft(x, -1), np.fft.fft(x), rtol=0, atol=1e-10 * n)
    assert np.allclose(oracle.dft(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-10 * n)


def test_fft_large_matches_numpy():
    n = 1 << 18
    x = _rand(n, 3)
    a = oracle.fft(x, +1)
    b = np.fft.ifft(x) * n
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(b))


def test_fft_closed_forms():
    n = 512
    # a delta at m transforms to exp(sign 2 pi i k m / n)
    m = 37
    x = np.zeros(n, complex)
    x[m] = 1.0
    k = np.arange(n)
    assert np.allclose(oracle.fft(x, +1), np.exp(2j * np.pi * k * m / n), atol=1e-13)
    assert np.allclose(oracle.fft(x, -1), np.exp(-2j * np.pi * k * m / n), atol=1e-13)
    # a pure tone exp(+2 pi i q j / n) becomes n * delta_{k,q} under sign -1
    q = 101
    tone = np.exp(2j * np.pi * q * np.arange(n) / n)
    y = oracle.fft(tone, -1)
    want = np.zeros(n, complex)
    want[q] = n
    assert np.allclose(y, want, atol=1e-10)


def test_fft_parseval():
    n = 1 << 14
    x = _rand(n, 11)
    y = oracle.fft(x, +1)
    assert np.isclose(np.sum(np.abs(y) ** 2), n * np.sum(np.abs(x) ** 2), rtol=1e-12)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.ones(12), 1)


def test_segment_spectrum_matches_numpy_rfft():
    n, fs = 1 << 16, 4096.0
    d = np.random.default_rng(5).standard_normal(n) * 1e-21
    got = oracle.segment_spectrum(d, fs)
    want = np.fft.rfft(d) / fs
    assert got.shape == (n // 2 + 1,)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
