"""Pins of the oracle's windowed output -- Eq. (impl-corr) at window starts n0 = k * hop,
window-local phase -- to a closed form, to the block's sliding-window recursion, and to
the whole-stream estimate (CPU only)."""
import math

import numpy as np
import pytest

import oracle
import synth


def g0(nu, N):
    """(1/N) sum_{n=0}^{N-1} exp(-j 2 pi nu n)."""
    nu = math.fmod(float(nu), 1.0)
    w = np.exp(-2j * np.pi * nu)
    if abs(w - 1.0) < 1e-15:
        return 1.0
    return (1.0 - np.exp(-2j * np.pi * math.fmod(nu * N, 1.0))) / (N * (1.0 - w))


def test_two_tones_per_window():
    """x, y tones f1, f2: window k gives exp(j 2 pi f1 m) exp(j 2 pi (f1 -+ f2) s_k) G0(a - f1 +- f2),
    s_k = k hop + M^- the window's first reference sample."""
    T, f1, f2, N, hop = 400, 0.1371, 0.0419, 64, 24
    lags = np.array([-5, 0, 3, 9])
    x, y = synth.tone(T, f1), synth.tone(T, f2)
    alphas = np.array([f1 - f2, f1 + f2, 0.0, -0.3])
    R = oracle.windows(x, y, lags, alphas, N, hop)
    assert R.shape[0] == (T - (5 + 9 + N)) // hop + 1
    for k in range(R.shape[0]):
        s = k * hop + 5
        for fi, sg in ((0, -1), (1, +1)):            # CONV: f1 - f2, CONJ: f1 + f2
            fd = f1 + sg * f2
            for ia, a in enumerate(alphas):
                G = g0(a - fd, N)
                for im, m in enumerate(lags):
                    ref = np.exp(2j * np.pi * f1 * m) * np.exp(2j * np.pi * math.fmod(fd * s, 1.0)) * G
                    assert abs(R[k, fi, ia, im] - ref) < 1e-11


def test_sliding_recursion_of_the_block_state():
    """hop = 1: N R_{k+1} = exp(j 2 pi a) (N R_k - p(s_k) + p(s_k + N) exp(-j 2 pi a N)), p(i) the
    lag product at reference sample i -- the update the block's `state` variable carries."""
    T, N = 300, 50
    x, y = synth.white(T, seed=20), synth.white(T, seed=21)
    lags, alphas = np.array([-2, 0, 4]), np.array([0.13, -0.41])
    R = oracle.windows(x, y, lags, alphas, N, 1)
    Mneg = 2
    for fi, conj in ((0, True), (1, False)):
        for ia, a in enumerate(alphas):
            for im, m in enumerate(lags):
                p = lambda i: x[i + m] * (np.conj(y[i]) if conj else y[i])
                for k in range(0, R.shape[0] - 1, 17):
                    s = k + Mneg
                    nxt = np.exp(2j * np.pi * a) * (N * R[k, fi, ia, im] - p(s) + p(s + N) * np.exp(-2j * np.pi * a * N))
                    assert abs(N * R[k + 1, fi, ia, im] - nxt) < 1e-10


def test_one_window_is_the_stream_estimate_with_its_phase_origin_moved():
    T = 257
    x = synth.white(T, seed=22)
    lags, alphas = np.array([-3, 1, 6]), np.array([0.0, 0.2, 0.37])
    N = T - 9
    R = oracle.windows(x, None, lags, alphas, N, 5)
    assert R.shape[0] == 1
    Rs, neff = oracle.estimate_xy(x, None, lags, alphas)
    assert neff == N
    rot = np.exp(2j * np.pi * np.asarray(alphas) * 3)[None, :, None]   # phase origin M^- = 3
    assert np.max(np.abs(R[0] - Rs * rot)) < 1e-12


@pytest.mark.parametrize("N,hop", [(16, 16), (32, 7), (8, 1)])
def test_full_grid_window_is_the_fft_of_the_lag_products(N, hop):
    """Full mode per window (Sec. 4: one FFT per lag over each window): on the grid
    a_kk = -1/2 + kk/N the windowed estimate is (1/N) FFT_N of p(n) (-1)^n, p the window's lag
    products -- numpy's FFT, independent of the oracle's direct sum."""
    T = 200
    x, y = synth.white(T, seed=23), synth.white(T, seed=24)
    lags = np.array([-3, 0, 2, 5])
    grid = -0.5 + np.arange(N) / N
    R = oracle.windows(x, y, lags, grid, N, hop)
    Mneg, sgn = 3, (-1.0) ** np.arange(N)
    assert R.shape[0] == (T - (3 + 5 + N)) // hop + 1
    for k in range(0, R.shape[0], 3):
        s = k * hop + Mneg
        for fi, conj in ((0, True), (1, False)):
            for im, m in enumerate(lags):
                yy = y[s:s + N]
                p = x[s + m:s + m + N] * (np.conj(yy) if conj else yy)
                ref = np.fft.fft(p * sgn) / N
                assert np.max(np.abs(R[k, fi, :, im] - ref)) < 1e-12
