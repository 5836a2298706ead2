"""Pins of the oracle's cyclic spectrum (the DFT over lags of a cyclic correlation estimate,
with a rectangular or Hann lag window), CPU only: a tone's line in closed form, Parseval
over lags distinct modulo Q, and the window's values."""
import numpy as np

import oracle
import synth


def test_tone_line_closed_form():
    """x = exp(j 2 pi f0 n): R^0(m) = exp(j 2 pi f0 m) exactly (CONV, a = 0), so the rectangular
    spectrum is sum_m exp(j 2 pi (f0 - f_q) m): L at f_q = f0, the Dirichlet sum elsewhere."""
    f0, Q = 0.125, 64
    lags = np.arange(-10, 11)
    x = synth.tone(2000, f0)
    R, _ = oracle.estimate_xy(x, None, lags, [0.0], forms=1)
    assert np.max(np.abs(R[0, 0] - np.exp(2j * np.pi * f0 * lags))) < 1e-12
    S = oracle.spectrum(R, lags, Q)
    fq = -0.5 + np.arange(Q) / Q
    ref = np.array([np.sum(np.exp(2j * np.pi * (f0 - f) * lags)) for f in fq])
    assert np.max(np.abs(S[0, 0] - ref)) < 1e-10
    assert np.argmax(np.abs(S[0, 0])) == int(round((f0 + 0.5) * Q))
    assert abs(np.max(np.abs(S[0, 0])) - len(lags)) < 1e-10


def test_parseval_over_lags_distinct_modulo_q():
    rng = np.random.default_rng(3)
    lags = np.array([-7, -3, 0, 1, 2, 9, 12])
    R = rng.normal(size=(2, 3, lags.size)) + 1j * rng.normal(size=(2, 3, lags.size))
    for Q in (32, 20):                                   # lags span 19 < Q: distinct mod Q
        for taper in (0, 1):
            S = oracle.spectrum(R, lags, Q, taper)
            w = oracle.lag_window(lags, taper)
            assert np.allclose(np.sum(np.abs(S) ** 2, axis=2), Q * np.sum(np.abs(R * w) ** 2, axis=2))


def test_hann_lag_window():
    w = oracle.lag_window([-4, 0, 4, 2], 1)
    assert np.allclose(w, [0.5 + 0.5 * np.cos(np.pi * 4 / 5), 1.0, 0.5 + 0.5 * np.cos(np.pi * 4 / 5),
                           0.5 + 0.5 * np.cos(np.pi * 2 / 5)])
    assert np.all(oracle.lag_window([-3, 5], 0) == 1.0)
