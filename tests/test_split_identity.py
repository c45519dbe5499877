"""The four-way frequency split that pass 2 uses for 16384-point rows (N = 2^22):
with b = b' + 4096 m and d = 4 k + q,
    z[4 k + q] = sum_b' exp(2 pi i b' k / 4096) u_q[b'],
    u_q[b'] = exp(2 pi i q b' / 16384) sum_m i^(m q) x[b' + 4096 m],
checked here in FP64 against the direct transform z[d] = sum_b x[b] exp(2 pi i b d / L),
together with the sample that output k of team (q0) lane l stands for:
c + n1 (q0 + 2 l) + 4 n1 k, i.e. c + n1 d."""

import numpy as np

L, Q = 16384, 4
M = L // Q


def _split(x):
    b = np.arange(M)
    xs = x.reshape(Q, M)  # xs[m, b'] = x[b' + 4096 m]
    out = np.empty((Q, M), dtype=complex)
    for q in range(Q):
        u = np.exp(2j * np.pi * q * b / L) * sum((1j ** (m * q)) * xs[m] for m in range(Q))
        out[q] = M * np.fft.ifft(u)  # sum_b' u[b'] exp(+2 pi i b' k / M)
    return out


def test_split_equals_the_direct_transform():
    rng = np.random.default_rng(20220)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    z = L * np.fft.ifft(x)  # z[d] = sum_b x[b] exp(+2 pi i b d / L)
    parts = _split(x)
    for q in range(Q):
        np.testing.assert_allclose(parts[q], z[q::Q], rtol=0, atol=1e-9 * np.abs(z).max())
    # a plain DFT sum at a few outputs, independent of numpy's FFT sign convention
    for d in (0, 1, 4097, L - 1):
        direct = np.sum(x * np.exp(2j * np.pi * np.arange(L) * d / L))
        assert abs(parts[d % Q][d // Q] - direct) < 1e-8 * np.abs(z).max()


def test_team_lanes_map_to_row_samples():
    # team 0 holds q = 0, 2 and team 1 q = 1, 3 as lanes l = 0, 1: q = q0 + 2 l
    n1, c = 256, 37
    for q0 in (0, 1):
        for l in (0, 1):
            q = q0 + 2 * l
            for k in (0, 1, 2047, M - 1):
                s = (c + q0 * n1) + l * (4 * n1 // 2) + 4 * n1 * k
                assert s == c + n1 * (4 * k + q)
