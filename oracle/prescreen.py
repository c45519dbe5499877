"""FP64 reference of the learned prescreen -- TEST INFRASTRUCTURE ONLY.

Only the tests may import this module; the CUDA library never does.  It
restates, in plain numpy, what the prescreen computes (the build's answer to
the paper's remark that at ~10^6 templates a brute-force search "is not the
best solution", Sec. introduction footnote):

* features: the whitened one-sided spectrum u_k = d~_k sqrt(4 df / S_k) on
  [f_low, fs/2) is split into B log-spaced bands; each band's analytic signal
  X_b(j) = sum_{k in band} u_k exp(+2 pi i j k / N) (a direct inverse DFT) is
  averaged in power over frames of F samples and normalised by its noise
  expectation 2 n_b; the feature is log of that ratio;
* network: conv1d(B -> 32, k 5, stride 1) -> ReLU -> 3 x [conv1d(32 -> 32, k 5,
  stride 2) -> ReLU] -> per-channel mean and max over time -> linear 64 -> 128
  -> ReLU -> linear 128 -> R; zero padding 2 on every convolution
  (out[o, t] = b[o] + sum_{i,k} W[o, i, k] in[i, s t + k - 2]);
* loss: soft-label cross entropy, mean over the batch;
* gradients by hand-written reverse-mode differentiation, pinned in the tests
  by central finite differences;
* the optimiser step: Adam with bias correction (Kingma and Ba, "Adam: a
  method for stochastic optimization", ICLR 2015, Algorithm 1);
* feature standardisation: per-band mean and population standard deviation
  over a set of feature rows, applied as (x - mean) / std before the network;
* ensemble scores: the mean over networks of their softmax probabilities.

Parameters travel as one flat vector in the order conv1.W, conv1.b, conv2.W,
conv2.b, conv3.W, conv3.b, conv4.W, conv4.b, fc1.W, fc1.b, fc2.W, fc2.b
(row-major shapes [32,B,5], [32], [32,32,5], [32], ..., [128,64], [128],
[R,128], [R]).
"""

from __future__ import annotations

import math

import numpy as np

CH = 32
KS = 5
HID = 128


def shapes(bands: int = 8, regions: int = 100):
    s = []
    cin = bands
    for _ in range(4):
        s += [(CH, cin, KS), (CH,)]
        cin = CH
    s += [(HID, 2 * CH), (HID,), (regions, HID), (regions,)]
    return s


def n_params(bands: int = 8, regions: int = 100) -> int:
    return sum(int(np.prod(x)) for x in shapes(bands, regions))


def unpack(theta, bands: int = 8, regions: int = 100):
    out, off = [], 0
    for shp in shapes(bands, regions):
        n = int(np.prod(shp))
        out.append(np.asarray(theta[off:off + n], dtype=np.float64).reshape(shp))
        off += n
    return out


def band_edges(n: int, fs: float, f_low: float, bands: int):
    """Bin ranges [k0, k1) of B log-spaced bands between f_low and fs/2."""
    df = fs / n
    edges = f_low * (fs / 2 / f_low) ** (np.arange(bands + 1) / bands)
    k = np.ceil(edges / df).astype(np.int64)
    k[0] = max(k[0], 1)
    k[-1] = n // 2
    return [(int(k[b]), int(k[b + 1])) for b in range(bands)]


def features(dtilde, psd, n: int, fs: float, f_low: float, bands: int = 8, frame: int = 512):
    """F[b, m] = log( mean_{j in frame m} |X_b(j)|^2 / (2 n_b) ), shape [B, n/frame]."""
    df = fs / n
    out = np.zeros((bands, n // frame))
    for b, (k0, k1) in enumerate(band_edges(n, fs, f_low, bands)):
        if k1 <= k0:
            continue
        k = np.arange(k0, k1)
        u = np.asarray(dtilde)[k0:k1] * np.sqrt(4.0 * df / np.asarray(psd)[k0:k1])
        j = np.arange(n)
        # direct inverse DFT of the band (no FFT), in blocks to bound memory
        x = np.zeros(n, dtype=np.complex128)
        for s in range(0, len(k), 256):
            kk = k[s:s + 256]
            x += np.exp(2j * np.pi * np.outer(j, kk) / n) @ u[s:s + 256]
        p = (np.abs(x) ** 2).reshape(n // frame, frame).mean(axis=1)
        out[b] = np.log(p / (2.0 * (k1 - k0)))
    return out


def _conv(x, W, b, stride):
    cin, L = x.shape
    co, _, ks = W.shape
    Lo = (L + 4 - ks) // stride + 1
    xp = np.zeros((cin, L + 4))
    xp[:, 2:2 + L] = x
    out = np.zeros((co, Lo))
    for t in range(Lo):
        out[:, t] = np.einsum("oik,ik->o", W, xp[:, stride * t:stride * t + ks]) + b
    return out


def forward(theta, x, bands: int = 8, regions: int = 100):
    """Logits and the activations of one sample x [B, T]."""
    P = unpack(theta, bands, regions)
    acts = [np.asarray(x, dtype=np.float64)]
    a = acts[0]
    for layer in range(4):
        W, b = P[2 * layer], P[2 * layer + 1]
        a = np.maximum(_conv(a, W, b, 1 if layer == 0 else 2), 0.0)
        acts.append(a)
    p = np.concatenate([a.mean(axis=1), a.max(axis=1)])
    h = np.maximum(P[8] @ p + P[9], 0.0)
    z = P[10] @ h + P[11]
    return z, dict(acts=acts, p=p, h=h)


def softmax(z):
    e = np.exp(z - z.max())
    return e / e.sum()


def loss(theta, xs, ys, bands: int = 8, regions: int = 100) -> float:
    tot = 0.0
    for x, y in zip(xs, ys):
        z, _ = forward(theta, x, bands, regions)
        lse = z.max() + math.log(np.exp(z - z.max()).sum())
        tot += -float(np.dot(y, z - lse))
    return tot / len(xs)


def _conv_back(x, W, dout, stride):
    """Gradients of out = conv(x) w.r.t. W, b and x given dout."""
    cin, L = x.shape
    co, _, ks = W.shape
    xp = np.zeros((cin, L + 4))
    xp[:, 2:2 + L] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for t in range(dout.shape[1]):
        seg = xp[:, stride * t:stride * t + ks]
        dW += np.einsum("o,ik->oik", dout[:, t], seg)
        dxp[:, stride * t:stride * t + ks] += np.einsum("o,oik->ik", dout[:, t], W)
    return dW, dout.sum(axis=1), dxp[:, 2:2 + L]


def gradient(theta, xs, ys, bands: int = 8, regions: int = 100):
    """d loss / d theta (flat), by reverse-mode differentiation."""
    P = unpack(theta, bands, regions)
    G = [np.zeros_like(q) for q in P]
    for x, y in zip(xs, ys):
        z, c = forward(theta, x, bands, regions)
        dz = softmax(z) * y.sum() - y  # d/dz of -sum_c y_c log softmax(z)_c
        G[10] += np.outer(dz, c["h"])
        G[11] += dz
        dh = (P[10].T @ dz) * (c["h"] > 0)
        G[8] += np.outer(dh, c["p"])
        G[9] += dh
        dp = P[8].T @ dh
        a4 = c["acts"][4]
        T = a4.shape[1]
        da = np.repeat((dp[:CH] / T)[:, None], T, axis=1)
        am = a4.argmax(axis=1)  # first maximum
        da[np.arange(CH), am] += dp[CH:]
        for layer in (3, 2, 1, 0):
            a_out = c["acts"][layer + 1]
            da = da * (a_out > 0)
            dW, db, dx = _conv_back(c["acts"][layer], P[2 * layer], da, 1 if layer == 0 else 2)
            G[2 * layer] += dW
            G[2 * layer + 1] += db
            da = dx
    return np.concatenate([g.ravel() for g in G]) / len(xs)


def soft_labels(region: int, regions: int = 100):
    """1 on the region of the injected chirp mass, 0.5 on its neighbours,
    normalised to sum 1."""
    y = np.zeros(regions)
    y[region] = 1.0
    if region > 0:
        y[region - 1] = 0.5
    if region < regions - 1:
        y[region + 1] = 0.5
    return y / y.sum()


def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def regions_of_bank(m1, m2, regions: int = 100):
    """Bank indices sorted by chirp mass, split into `regions` equal-count
    groups; returns (list of index arrays, chirp-mass boundaries)."""
    mc = chirp_mass(m1, m2)
    order = np.argsort(mc, kind="stable")
    groups = np.array_split(order, regions)
    bounds = np.array([mc[g[-1]] for g in groups[:-1]])
    return groups, bounds


def region_of(mc, bounds) -> int:
    return int(np.searchsorted(bounds, mc, side="left"))


def adam_step(theta, m, v, g, step: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam update at step t = `step` (1 for the first), FP64:
    m_t = b1 m + (1 - b1) g;  v_t = b2 v + (1 - b2) g^2;
    m^ = m_t / (1 - b1^t);  v^ = v_t / (1 - b2^t);
    theta_t = theta - lr m^ / (sqrt(v^) + eps).
    Returns (theta_t, m_t, v_t)."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m_t = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v_t = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    m_hat = m_t / (1.0 - beta1 ** step)
    v_hat = v_t / (1.0 - beta2 ** step)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m_t, v_t


def fit_norm(feats):
    """Per-band mean and population standard deviation of feature rows
    [count, B, T] over count * T values; a zero spread reads 1."""
    f = np.asarray(feats, dtype=np.float64)
    mean = f.mean(axis=(0, 2))
    sd = np.sqrt(np.maximum(((f - mean[None, :, None]) ** 2).mean(axis=(0, 2)), 0.0))
    return mean, np.where(sd > 0, sd, 1.0)


def standardise(x, mean, sd):
    """(x - mean_b) / sd_b for one feature row [B, T]."""
    return (np.asarray(x, dtype=np.float64) - np.asarray(mean)[:, None]) / np.asarray(sd)[:, None]


def ensemble_probabilities(logit_rows):
    """Mean over networks of softmax(z): logit_rows [k][R] -> [R]."""
    return np.mean([softmax(np.asarray(z, dtype=np.float64)) for z in logit_rows], axis=0)
