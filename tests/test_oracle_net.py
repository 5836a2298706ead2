"""Pins of the FP64 proposer oracle (CPU): explicit-loop convolution, finite-difference
gradients, closed-form BCE values, and the line positions of a tone's features."""
import math

import numpy as np
import pytest

from oracle import net as on


def test_conv_matches_explicit_loops():
    rng = np.random.default_rng(0)
    ci, co, n = 3, 4, 20
    x = rng.normal(size=(ci, n))
    W = rng.normal(size=(co, ci, on.K))
    b = rng.normal(size=co)
    y = on.conv(x, W, b)
    for o in range(co):
        for i in range(n):
            ref = b[o] + sum(W[o, c, k] * x[c, (i + k - 4) % n] for c in range(ci) for k in range(on.K))
            assert abs(y[o, i] - ref) < 1e-12


def test_conv_backward_finite_differences():
    rng = np.random.default_rng(1)
    ci, co, n = 3, 5, 24
    x = rng.normal(size=(ci, n))
    W = rng.normal(size=(co, ci, on.K))
    b = rng.normal(size=co)
    gy = rng.normal(size=(co, n))
    L = lambda x_, W_, b_: float(np.sum(gy * on.conv(x_, W_, b_)))
    dx, dW, db = on.conv_backward(x, W, gy)
    eps = 1e-6
    for (c, j) in [(0, 0), (2, 23), (1, 7)]:
        xp, xm = x.copy(), x.copy()
        xp[c, j] += eps
        xm[c, j] -= eps
        assert abs((L(xp, W, b) - L(xm, W, b)) / (2 * eps) - dx[c, j]) < 1e-6
    for (o, c, k) in [(0, 0, 0), (4, 2, 8), (2, 1, 4)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[o, c, k] += eps
        Wm[o, c, k] -= eps
        assert abs((L(x, Wp, b) - L(x, Wm, b)) / (2 * eps) - dW[o, c, k]) < 1e-6
    assert np.allclose(db, gy.sum(axis=1))


def test_bce_closed_forms():
    z = np.array([[0.0, 2.0], [-3.0, 0.5]])
    y = np.array([[1.0, 0.0], [1.0, 1.0]])
    loss, g = on.bce(z, y, pos_weight=2.0)
    s = 1 / (1 + np.exp(-z))
    ref = np.mean(2.0 * y * -np.log(s) + (1 - y) * -np.log(1 - s))
    assert abs(loss - ref) < 1e-12
    assert abs(on.bce(np.zeros(4), np.zeros(4))[0] - math.log(2.0)) < 1e-15
    assert np.allclose(g, (2.0 * y * (s - 1) + (1 - y) * s) / z.size)


@pytest.mark.slow
def test_full_net_gradient_finite_differences():
    params = on.init_params(3)
    rng = np.random.default_rng(2)
    feat = rng.normal(size=(on.NIN, on.NFFT))
    lab = (rng.uniform(size=(2, on.NBIN)) < 0.05).astype(float)
    loss, grads = on.batch_loss_and_grads(params, [feat], [lab], pos_weight=3.0)
    eps = 1e-5
    for (li, idx) in [(0, (5, 1, 3)), (2, (10, 20, 4)), (3, (1, 63, 8))]:
        W, b = params[li]
        Wp = [(w.copy(), bb.copy()) for w, bb in params]
        Wm = [(w.copy(), bb.copy()) for w, bb in params]
        Wp[li][0][idx] += eps
        Wm[li][0][idx] -= eps
        lp, _ = on.batch_loss_and_grads(Wp, [feat], [lab], pos_weight=3.0)
        lm, _ = on.batch_loss_and_grads(Wm, [feat], [lab], pos_weight=3.0)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grads[li][0][idx]) < 1e-6 * max(1.0, abs(fd)) + 1e-9, (li, idx)


def test_tone_feature_lines():
    """x = exp(j 2 pi f0 n): the x channel peaks at f0, x^2 at 2 f0, and every lag product
    x[n+d] x*[n] = exp(j 2 pi f0 d) is constant: its line is at 0."""
    f0 = 0.1171875                                   # on the 4096-bin grid: 480/4096
    n = np.arange(on.NEED)
    x = np.exp(2j * np.pi * f0 * n)
    F = on.features(x)
    j = lambda f: int(round((f + 0.5) * on.NFFT)) % on.NFFT
    assert F.shape == (on.NIN, on.NFFT)
    assert int(np.argmax(F[0])) == j(f0)
    assert int(np.argmax(F[1])) == j(2 * f0)
    for c in range(2, on.NIN):
        assert int(np.argmax(F[c])) == j(0.0)


def test_lag_product_channel_shows_a_conventional_line():
    """Rectangular BPSK at 8 samples/symbol: the lag-4 product has a line at 1/8 (its cyclic
    autocorrelation at lag 4 is nonzero at the baud rate), the |x|^2 channel has none."""
    import synth
    x = synth.rect_bpsk(on.NEED, sps=8, seed=5)
    F = on.features(x)
    j = lambda f: int(round((f + 0.5) * on.NFFT)) % on.NFFT
    c4 = 2 + on.LAG_CHANNELS.index(4)
    k = j(0.125)
    assert F[c4, k] > 3.0 and F[c4, k] > np.median(F[c4]) + 3.0
    assert F[c4, k] > F[c4, k - 5] + 2.0 and F[c4, k] > F[c4, k + 5] + 2.0
    assert abs(F[2, k] - np.median(F[2])) < 1e-6     # |x|^2 = 1: no line at 1/8
    assert np.allclose(F.mean(axis=1), 0.0, atol=1e-9) and np.allclose(F.std(axis=1), 1.0, atol=1e-9)


def test_welch_hann_tone_closed_form():
    """A bin-centred tone A exp(j 2 pi k0 n / N) under the Hann window w = 1/2 - 1/2 cos(2 pi n / N):
    the windowed DFT is A N (1/2 at k0, -1/4 at k0 +- 1, 0 elsewhere), so the periodogram has
    exactly three non-zero bins A^2 N^2 (1/16, 1/4, 1/16) -- ratios 1:4:1 -- and every segment
    is the same, so the 16-segment mean equals one of them.  x^2 is the tone 2 k0 with A^2, and
    a lag product x[n+d] conj(x[n]) = A^2 exp(j 2 pi k0 d / N) is a constant: its three bins
    are at 0 and +-1.  (A rectangular window would give one bin; a wrong segment count or
    scaling another level.)"""
    N, k0, amp = on.NFFT, 37, 0.75
    x = amp * np.exp(2j * np.pi * k0 * np.arange(on.NEED) / N)
    P = on.welch(x)
    for c, (k, a2) in enumerate([(k0, amp ** 2), (2 * k0, amp ** 4)] + [(0, amp ** 4)] * len(on.LAG_CHANNELS)):
        expect = np.zeros(N)
        expect[k % N] = a2 * N * N / 4
        expect[(k + 1) % N] = expect[(k - 1) % N] = a2 * N * N / 16
        assert np.allclose(P[c], expect, rtol=1e-9, atol=1e-9 * a2 * N * N), c


def test_welch_averages_the_segments():
    """Segments with different amplitudes: the Welch estimate is the mean of their periodograms
    (sum of the squared amplitudes over the 16 segments, divided by 16)."""
    N, k0 = on.NFFT, 100
    amps = 1.0 + 0.25 * np.arange(on.NSEG)
    n = np.arange(on.NEED)
    a = np.concatenate([np.repeat(amps, N), np.full(on.NEED - on.NSEG * N, amps[-1])])
    x = a * np.exp(2j * np.pi * k0 * n / N)
    P = on.welch(x)
    assert abs(P[0, k0] - np.mean(amps ** 2) * N * N / 4) < 1e-9 * P[0, k0]


def test_features_are_the_standardised_log_of_the_shifted_welch_spectrum():
    """features = per channel (L - mean L) / std L with L = log10(Welch + 1e-12), frequency bins
    shifted so that bin j is -1/2 + j/N: checked through properties that pin each step -- the
    shift (a tone's peak bin), the standardisation (zero mean, unit spread), and the log
    (a scaled signal gives the same features for x, whose spectrum has no floor)."""
    import synth
    x = synth.white(on.NEED, seed=11)
    F = on.features(x)
    G = on.features(3.0 * x)
    assert np.allclose(F.mean(axis=1), 0.0, atol=1e-9) and np.allclose(F.std(axis=1), 1.0, atol=1e-9)
    assert np.allclose(F[0], G[0], atol=1e-9)                     # log10(9 P) - mean: the 9 cancels
    P = on.welch(x)
    L = np.log10(np.roll(P, on.NFFT // 2, axis=1) + 1e-12)
    assert np.allclose(np.corrcoef(F[0], L[0])[0, 1], 1.0, atol=1e-12)
