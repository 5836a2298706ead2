"""Pins of the oracle's full Eq. (impl-corr) form -- two inputs x, y and signed lags
m in [-M^-, M^+] -- to closed forms and to a brute-force matrix product (CPU only).

A slip in the cross form (y and x swapped, the conjugate on the wrong input, the window
not starting M^- samples in, the phase referred to the x sample instead of the y sample,
N_eff not T - M^- - M^+) fails one of these."""
import math

import numpy as np
import pytest

import oracle
import synth

CONV, CONJ = oracle.CONV, oracle.CONJ


def geometric_mean(nu, N, start):
    """(1/N) sum_{n=start}^{start+N-1} exp(-j 2 pi nu n), summed in closed form."""
    nu = math.fmod(float(nu), 1.0)
    w = np.exp(-2j * np.pi * nu)
    lead = np.exp(-2j * np.pi * math.fmod(nu * start, 1.0))
    if abs(w - 1.0) < 1e-15:
        return lead
    return lead * (1.0 - np.exp(-2j * np.pi * math.fmod(nu * N, 1.0))) / (N * (1.0 - w))


@pytest.mark.parametrize("n0", [0, 12345])
def test_two_tones_closed_form(n0):
    """x = exp(j 2 pi f1 n), y = exp(j 2 pi f2 n) (absolute n):
    CONV R[a][m] = exp(j 2 pi f1 m) G(a - f1 + f2), CONJ R[a][m] = exp(j 2 pi f1 m) G(a - f1 - f2),
    G(nu) the mean of exp(-j 2 pi nu n) over n = n0 + M^- .. n0 + M^- + N_eff - 1."""
    T, f1, f2 = 700, 0.1234, -0.0771
    lags = np.array([-9, -3, 0, 2, 11])
    Mneg, Mpos = 9, 11
    x = synth.tone(T, f1, n_start=n0)
    y = synth.tone(T, f2, n_start=n0)
    alphas = np.array([f1 - f2, f1 + f2, 0.0, 0.31, -0.45])
    R, neff = oracle.estimate_xy(x, y, lags, alphas, n0=n0)
    assert neff == T - Mneg - Mpos
    for fi, sgn in ((0, +1), (1, -1)):              # CONV: nu = a - f1 + f2; CONJ: nu = a - f1 - f2
        for ia, a in enumerate(alphas):
            G = geometric_mean(a - f1 + sgn * f2, neff, n0 + Mneg)
            for im, m in enumerate(lags):
                ref = np.exp(2j * np.pi * f1 * m) * G
                assert abs(R[fi, ia, im] - ref) < 1e-11, (fi, a, m)


def test_brute_force_matrix_form_signed_lags_cross():
    """R = P^T w / N_eff with P[n][m] = x[n+m] c(y[n]) built row by row over the committed
    n-range and w[n] = exp(-j 2 pi a n) from an exact rational phase."""
    from fractions import Fraction
    T = 53
    rng = np.random.default_rng(5)
    x = rng.normal(size=T) + 1j * rng.normal(size=T)
    y = rng.normal(size=T) + 1j * rng.normal(size=T)
    lags = [4, -6, 0, -1, 4, 9]
    alphas = [Fraction(3, 17), Fraction(-5, 11), Fraction(0)]
    R, neff = oracle.estimate_xy(x, y, lags, [float(a) for a in alphas])
    Mneg, Mpos = 6, 9
    assert neff == T - Mneg - Mpos
    ns = list(range(Mneg, T - Mpos))
    for fi, conj in ((0, True), (1, False)):
        P = np.array([[x[n + m] * (np.conj(y[n]) if conj else y[n]) for m in lags] for n in ns])
        for ia, a in enumerate(alphas):
            w = np.array([np.exp(-2j * np.pi * float((a * n) % 1)) for n in ns])
            ref = (w @ P) / len(ns)
            assert np.max(np.abs(R[fi, ia] - ref)) < 1e-12


def test_reduces_to_the_auto_estimator():
    """y = x (passed explicitly or as None) with lags >= 0 is the cyclic ACF/CCF estimate."""
    x = synth.white(300, seed=9)
    lags, alphas = [0, 2, 7], [0.0, 0.123, -0.4]
    R0, n0 = oracle.estimate(x, lags, alphas)
    R1, n1 = oracle.estimate_xy(x, None, lags, alphas)
    R2, n2 = oracle.estimate_xy(x, x.copy(), lags, alphas)
    assert n0 == n1 == n2 == 293
    assert np.array_equal(R0, R1) and np.array_equal(R0, R2)


def test_negative_lags_shift_the_window():
    """Lags all <= 0 of x against itself: R[m] for m = -k equals the auto estimate of the
    reversed roles, x[n-k] conj(x[n]) summed over n = k .. T-1, i.e. conj of the lag-k
    product summed over n' = n - k = 0 .. T-1-k with the phase at n' + k."""
    T = 200
    x = synth.white(T, seed=11)
    a = 0.2
    R, neff = oracle.estimate_xy(x, None, [-5, 0], [a], forms=CONV)
    assert neff == T - 5
    n = np.arange(5, T)
    ref = np.mean(x[n - 5] * np.conj(x[n]) * np.exp(-2j * np.pi * a * n))
    assert abs(R[0, 0, 0] - ref) < 1e-12
    # the same terms read from the positive lag: conj(x[n'+5] conj(x[n'])) at phase n'+5
    n2 = np.arange(0, T - 5)
    ref2 = np.mean(np.conj(x[n2 + 5] * np.conj(x[n2])) * np.exp(-2j * np.pi * a * (n2 + 5)))
    assert abs(ref - ref2) < 1e-12


def test_r00_xy_is_the_cauchy_schwarz_bound():
    T = 400
    x = synth.white(T, seed=12) * 2.0
    y = synth.white(T, seed=13) * 0.5
    lags = [-7, 0, 3, 10]
    R, neff = oracle.estimate_xy(x, y, lags, [0.0, 0.17])
    b = oracle.r00_xy(x, y, 7, 10)
    n = np.arange(7, T - 10)
    assert abs(b - math.sqrt(np.mean(np.abs(x[n]) ** 2) * np.mean(np.abs(y[n]) ** 2))) < 1e-12
    assert np.all(np.abs(R[:, :, 1]) <= b * (1 + 1e-12))     # lag 0: |mean x[n] c(y[n]) w| <= b
    assert abs(oracle.r00_xy(x, None, 7, 10) - np.mean(np.abs(x[n]) ** 2)) < 1e-12
