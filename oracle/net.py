"""FP64 CPU oracle of the cycle-frequency proposer -- TEST INFRASTRUCTURE.

Only tests may import this module.  It restates, in plain numpy float64, what the GPU
proposer computes, so that the CUDA features, forward pass, gradients and loss can be
checked value by value:

* features(x): Welch-averaged periodograms (16 segments of 4096 samples, Hann window) of
  x, x**2 and of the lag products x[n+d] conj(x[n]) for d in LAG_CHANNELS (d = 0 is
  |x|^2) -- the spectra in which conjugate (x^2) and conventional (lag products) cycle
  frequencies show up as lines (Sec. 2: the cyclic statistics are Fourier coefficients of
  the lag products; a constant-envelope signal such as GMSK has its conventional lines at
  non-zero lags only) -- as log10, frequency axis shifted to [-1/2, 1/2), each channel
  standardised to zero mean and unit variance.  Needs 65536 + 16 samples.
* forward/backward of the net: four circular 1-D convolutions (kernel 9, padding 4),
  11 -> 64 -> 64 -> 64 -> 2 channels, ReLU after the first three, then the mean over
  groups of 8 bins: 2 x 512 logits, one per cycle-frequency grid bin a = -1/2 + k/512
  and form (CONV, CONJ).
* the loss: mean binary cross-entropy with logits, positives weighted by `pos_weight`.

The pins are in tests/test_oracle_net.py (finite differences, a direct DFT, closed cases).
"""
from __future__ import annotations

import numpy as np

NFFT, NSEG, NBIN, POOL, K = 4096, 16, 512, 8, 9
LAG_CHANNELS = (0, 1, 2, 3, 4, 6, 8, 12, 16)
NIN = 2 + len(LAG_CHANNELS)
CH = (NIN, 64, 64, 64, 2)
NEED = NSEG * NFFT + max(LAG_CHANNELS)


def hann(n: int = NFFT) -> np.ndarray:
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(n) / n)


def welch(x, nseg: int = NSEG, nfft: int = NFFT) -> np.ndarray:
    """[NIN][nfft] float64: the mean over nseg consecutive segments of nfft samples of the
    periodogram |FFT(y w)|^2 (Hann window w, no other scaling, FFT bin order) of each channel
    y: x, x^2 and the lag products x[n+d] conj(x[n])."""
    x = np.asarray(x, dtype=np.complex128)
    assert x.size >= nseg * nfft + max(LAG_CHANNELS)
    w = hann(nfft)
    out = np.zeros((NIN, nfft))
    for s in range(nseg):
        n = np.arange(s * nfft, (s + 1) * nfft)
        seg = x[n]
        ys = [seg, seg * seg] + [x[n + d] * np.conj(seg) for d in LAG_CHANNELS]
        for c, y in enumerate(ys):
            Y = np.fft.fft(y * w)
            out[c] += np.abs(Y) ** 2
    return out / nseg


def features(x, nseg: int = NSEG, nfft: int = NFFT, eps: float = 1e-12) -> np.ndarray:
    """[NIN][nfft] float64 standardised log spectra (see module doc)."""
    out = np.log10(welch(x, nseg, nfft) + eps)
    out = np.roll(out, nfft // 2, axis=1)                 # bin j <-> frequency -1/2 + j/nfft
    mu = out.mean(axis=1, keepdims=True)
    sd = out.std(axis=1, keepdims=True)
    return (out - mu) / np.maximum(sd, 1e-6)


def init_params(seed: int = 0):
    """He-normal weights, zero biases: list of (W[co][ci][K], b[co])."""
    rng = np.random.default_rng(seed)
    ps = []
    for ci, co in zip(CH[:-1], CH[1:]):
        ps.append((rng.normal(0.0, np.sqrt(2.0 / (ci * K)), (co, ci, K)), np.zeros(co)))
    return ps


def conv(x, W, b):
    """Circular 1-D convolution: y[co][i] = b[co] + sum_ci sum_k W[co][ci][k] x[ci][i+k-4]."""
    n = x.shape[-1]
    y = np.tile(b[:, None], (1, n)).astype(np.float64)
    for k in range(K):
        y += W[:, :, k] @ np.roll(x, -(k - K // 2), axis=-1)
    return y


def conv_backward(x, W, dy):
    """Gradients of conv(x, W, b) given dL/dy: (dL/dx, dL/dW, dL/db)."""
    dx = np.zeros_like(x, dtype=np.float64)
    dW = np.zeros_like(W, dtype=np.float64)
    for k in range(K):
        xs = np.roll(x, -(k - K // 2), axis=-1)
        dW[:, :, k] = dy @ xs.T
        dx += np.roll(W[:, :, k].T @ dy, k - K // 2, axis=-1)
    return dx, dW, dy.sum(axis=-1)


def forward(params, feat):
    """feat [3][4096] -> logits [2][512]; also returns the cache for backward."""
    h = [np.asarray(feat, dtype=np.float64)]
    pre = []
    for li, (W, b) in enumerate(params):
        z = conv(h[-1], W, b)
        pre.append(z)
        h.append(np.maximum(z, 0.0) if li < len(params) - 1 else z)
    logits = h[-1].reshape(2, NBIN, POOL).mean(axis=-1)
    return logits, (h, pre)


def bce(logits, labels, pos_weight: float = 1.0):
    """Mean over entries of  -[pw y log s(z) + (1-y) log(1-s(z))]  and dL/dlogits."""
    z = np.asarray(logits, dtype=np.float64)
    y = np.asarray(labels, dtype=np.float64)
    lsp = np.logaddexp(0.0, -z)                 # -log s(z)
    lsn = np.logaddexp(0.0, z)                  # -log(1 - s(z))
    loss = np.mean(pos_weight * y * lsp + (1.0 - y) * lsn)
    s = 1.0 / (1.0 + np.exp(-z))
    grad = (pos_weight * y * (s - 1.0) + (1.0 - y) * s) / z.size
    return loss, grad


def backward(params, cache, dlogits):
    """Parameter gradients [(dW, db), ...] given dL/dlogits [2][512]."""
    h, pre = cache
    dz = np.repeat(np.asarray(dlogits, dtype=np.float64), POOL, axis=-1) / POOL
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        if li < len(params) - 1:
            dz = dz * (pre[li] > 0.0)
        dx, dW, db = conv_backward(h[li], W, dz)
        grads[li] = (dW, db)
        dz = dx
    return grads


def batch_loss_and_grads(params, feats, labels, pos_weight: float = 1.0):
    """Mean loss over a batch (each sample's mean BCE, averaged) and its gradients."""
    B = len(feats)
    tot = 0.0
    acc = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    for f, y in zip(feats, labels):
        z, cache = forward(params, f)
        loss, g = bce(z, y, pos_weight)
        tot += loss / B
        gr = backward(params, cache, g / B)
        acc = [(aW + gW, ab + gb) for (aW, ab), (gW, gb) in zip(acc, gr)]
    return tot, acc
