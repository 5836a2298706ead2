"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics (CPU only).

Each test would fail on a plausible slip in the oracle: a dropped conjugate, a flipped
phase sign, lag and sample indices swapped, the wrong normaliser, the phase origin, or
a lossy a*n reduction.  None of them re-types the oracle's own formula.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CONV, CONJ = oracle.CONV, oracle.CONJ


def dirichlet(nu, N, n0=0):
    """(1/N) sum_{n=n0}^{n0+N-1} exp(-j 2 pi nu n), geometric-series closed form."""
    nu = float(nu)
    w = np.exp(-2j * np.pi * math.fmod(nu, 1.0))
    lead = np.exp(-2j * np.pi * math.fmod(nu * n0, 1.0)) if n0 else 1.0
    if abs(w - 1.0) < 1e-15:
        return lead
    wN = np.exp(-2j * np.pi * math.fmod(nu * N, 1.0))
    return lead * (1.0 - wN) / (N * (1.0 - w))


def rnd_complex(T, seed):
    return synth.white(T, seed=seed)


# ---------------------------------------------------------------------------------------
# Closed form: complex exponential (conjugate R at a = 2 f0 equals exp(j 2 pi f0 m))
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("f0", [0.05, -0.1875, 0.3141592653589793])
@pytest.mark.parametrize("n0", [0, 12345])
def test_tone_closed_form(f0, n0):
    T, lags = 700, np.array([0, 1, 5, 13, 2])
    M = lags.max()
    N = T - M
    x = synth.tone(T, f0, n_start=n0)
    al = np.array([0.0, 2 * f0, -2 * f0, 0.173, 2 * f0 + 1.0, 0.5, 1.0 / N])
    R, neff = oracle.estimate(x, lags, al, CONV | CONJ, n0=n0)
    assert neff == N
    for ia, a in enumerate(al):
        for im, m in enumerate(lags):
            lag_phase = np.exp(2j * np.pi * f0 * m)
            # conventional: x[n+m] x*[n] = exp(j 2 pi f0 m) -> lag phase times D(a)
            conv = lag_phase * dirichlet(a, N, n0)
            # conjugate: x[n+m] x[n] = exp(j 2 pi f0 m) exp(j 2 pi 2 f0 (n0 + n)) -> D(a - 2 f0)
            conj = lag_phase * dirichlet(a - 2 * f0, N, n0)
            assert abs(R[0, ia, im] - conv) < 1e-11, (a, m)
            assert abs(R[1, ia, im] - conj) < 1e-11, (a, m)
    # the benchmark spec itself: conjugate R at a = 2 f0 is exp(j 2 pi f0 m) (n0 = 0)
    if n0 == 0:
        assert np.allclose(R[1, 1, :], np.exp(2j * np.pi * f0 * lags), atol=1e-12)


# ---------------------------------------------------------------------------------------
# Special cases that reduce to a library routine (pocketfft through numpy)
# ---------------------------------------------------------------------------------------

def test_dft_of_lag_products():
    """At a = k/N_eff the estimator is the N_eff-point DFT of each lag-product sequence."""
    T, lags = 48, np.array([0, 2, 7, 3])
    N = T - lags.max()
    x = rnd_complex(T, 11)
    al = np.arange(N) / N
    R, _ = oracle.estimate(x, lags, al, CONV | CONJ)
    for im, m in enumerate(lags):
        p = x[m:m + N] * np.conj(x[:N])
        q = x[m:m + N] * x[:N]
        assert np.allclose(R[0, :, im], np.fft.fft(p) / N, atol=1e-13)
        assert np.allclose(R[1, :, im], np.fft.fft(q) / N, atol=1e-13)


def test_lag0_fft_of_power_and_square():
    T = 64
    x = rnd_complex(T, 12)
    al = np.arange(T) / T
    R, _ = oracle.estimate(x, [0], al, CONV | CONJ)
    assert np.allclose(R[0, :, 0], np.fft.fft(np.abs(x) ** 2) / T, atol=1e-13)
    assert np.allclose(R[1, :, 0], np.fft.fft(x * x) / T, atol=1e-13)


def test_brute_force_matrix_form():
    """Lag-product matrix times an explicit DFT matrix; unsorted lags with a duplicate."""
    T, lags = 60, np.array([5, 0, 3, 5, 9])
    N = T - lags.max()
    x = rnd_complex(T, 13)
    rng = np.random.default_rng(5)
    al = rng.uniform(-2.0, 2.0, 9)
    n = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(al, n))                  # [A][N]
    P = np.stack([x[m:m + N] * np.conj(x[:N]) for m in lags])  # [L][N]
    Q = np.stack([x[m:m + N] * x[:N] for m in lags])
    R, _ = oracle.estimate(x, lags, al, CONV | CONJ)
    assert np.allclose(R[0], E @ P.T / N, atol=1e-12)
    assert np.allclose(R[1], E @ Q.T / N, atol=1e-12)
    Rc, _ = oracle.estimate(x, lags, al, CONJ)                 # single form selects CONJ
    assert np.array_equal(Rc[0], R[1])


# ---------------------------------------------------------------------------------------
# Phase at large n
# ---------------------------------------------------------------------------------------

def exact_rot(a, n0):
    """exp(-j 2 pi a n0) with a*n0 reduced mod 1 in exact rational arithmetic."""
    f = (Fraction(a) * n0) % 1
    return np.exp(-2j * np.pi * float(f))


def test_time_shift_large_start_index():
    T, lags = 300, np.arange(6)
    x = rnd_complex(T, 14)
    al = np.array([0.1, -0.33, 0.123456789, 0.5, 1.0 / 3.0])
    n0 = (1 << 40) + 12345
    R0, _ = oracle.estimate(x, lags, al, CONV | CONJ, n0=0)
    R1, _ = oracle.estimate(x, lags, al, CONV | CONJ, n0=n0)
    for ia, a in enumerate(al):
        assert np.allclose(R1[:, ia, :], exact_rot(a, n0) * R0[:, ia, :], atol=1e-12)


def test_dyadic_cycle_frequencies_exact_integer_phase():
    T, lags = 200, np.array([0, 1, 4])
    N = T - 4
    x = rnd_complex(T, 15)
    ks = np.arange(-8, 8)
    R, _ = oracle.estimate(x, lags, ks / 8.0, CONV | CONJ, n0=1 << 45)
    roots = np.exp(-2j * np.pi * np.arange(8) / 8.0)
    n = np.arange(N, dtype=np.int64) + (1 << 45)
    for ik, k in enumerate(ks):
        w = roots[(k * n) % 8]
        for im, m in enumerate(lags):
            assert abs(R[0, ik, im] - np.sum(w * x[m:m + N] * np.conj(x[:N])) / N) < 1e-13
            assert abs(R[1, ik, im] - np.sum(w * x[m:m + N] * x[:N]) / N) < 1e-13


def test_aliasing_a_plus_integer():
    T = 150
    x = rnd_complex(T, 16)
    base = np.array([0.125, -0.40625, 0.0078125])               # dyadic: a + k is exact
    R0, _ = oracle.estimate(x, [0, 3], base, CONV | CONJ, n0=977)
    for k in (1, -3, 17):
        Rk, _ = oracle.estimate(x, [0, 3], base + k, CONV | CONJ, n0=977)
        assert np.allclose(Rk, R0, atol=1e-13)


# ---------------------------------------------------------------------------------------
# Streaming = batch on the concatenation: sums over adjacent n-ranges add
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("N1", [1, 17, 40])
def test_split_sums_add(N1):
    T, lags = 120, np.array([0, 7, 2])
    M = 7
    x = rnd_complex(T, 17)
    al = np.array([0.3, -0.11, 0.0])
    Rall, Nall = oracle.estimate(x, lags, al)
    Ra, Na = oracle.estimate(x[:N1 + M], lags, al)
    Rb, Nb = oracle.estimate(x[N1:], lags, al, n0=N1)
    assert Na == N1 and Na + Nb == Nall
    assert np.allclose(Rall * Nall, Ra * Na + Rb * Nb, atol=1e-11)


def test_empty_when_too_short():
    x = rnd_complex(5, 1)
    R, neff = oracle.estimate(x, [0, 5], [0.1])
    assert R is None and neff == 0
    with pytest.raises(ValueError):
        oracle.estimate(x, [-1, 2], [0.1])


# ---------------------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------------------

def test_conjugate_symmetry_lag0_and_scaling_and_cauchy_schwarz():
    T, lags = 257, np.arange(0, 9)
    N = T - 8
    x = rnd_complex(T, 18) + 0.3
    al = np.array([0.07, -0.07, 0.25, -0.25, 0.0])
    R, _ = oracle.estimate(x, lags, al)
    assert abs(R[0, 1, 0] - np.conj(R[0, 0, 0])) < 1e-13
    assert abs(R[0, 3, 0] - np.conj(R[0, 2, 0])) < 1e-13
    assert abs(R[0, 4, 0].imag) < 1e-14
    c = 0.7 - 1.3j
    Rs, _ = oracle.estimate(c * x, lags, al)
    assert np.allclose(Rs[0], abs(c) ** 2 * R[0], atol=1e-12)
    assert np.allclose(Rs[1], c * c * R[1], atol=1e-12)
    E0 = np.sum(np.abs(x[:N]) ** 2)
    for im, m in enumerate(lags):
        Em = np.sum(np.abs(x[m:m + N]) ** 2)
        assert np.all(np.abs(R[:, :, im]) <= math.sqrt(Em * E0) / N * (1 + 1e-12))


def test_r00_is_mean_power():
    x = rnd_complex(100, 19)
    assert abs(oracle.r00(x, 10) - np.mean(np.abs(x[:90]) ** 2)) < 1e-14
    assert abs(oracle.r00(x, 10) - oracle.estimate(x, [0, 10], [0.0], CONV)[0][0, 0, 0].real) < 1e-14


# ---------------------------------------------------------------------------------------
# Statistical pins (seeded; bands in units of R^0(0)/sqrt(N_eff))
# ---------------------------------------------------------------------------------------

def test_white_noise_statistics():
    T, lags = (1 << 14) + 7, np.arange(8)
    x = synth.white(T, seed=0xC7C1_0101)
    al = np.array([0.0, 0.01, 0.125, -0.3, 0.5, 0.2222])
    R, N = oracle.estimate(x, lags, al)
    band = 5.0 / math.sqrt(N)
    assert abs(R[0, 0, 0] - 1.0) < band
    mask = np.ones(R.shape, bool)
    mask[0, 0, 0] = False
    assert np.all(np.abs(R[mask]) < band)
    # E|R|^2 = 1/N for the zero-mean entries (mean over 95 entries, loose factor)
    assert 0.5 / N < np.mean(np.abs(R[mask]) ** 2) < 1.6 / N


def test_rect_bpsk_lines_at_baud_multiples():
    sps, T = 4, (1 << 15) + 5
    x = synth.rect_bpsk(T, sps=sps, seed=0xC7C1_0102)
    lags = np.arange(6)
    al = np.concatenate([np.arange(sps) / sps, [0.1, 0.37, -0.2]])
    R, N = oracle.estimate(x, lags, al)
    band = 5.0 / math.sqrt(N)
    for ia, a in enumerate(al):
        for im, m in enumerate(lags):
            if ia < sps:
                k = ia
                expect = sum(np.exp(-2j * np.pi * k * n / sps) for n in range(sps - m)) / sps if m < sps else 0.0
            else:
                expect = 0.0
            # a real-valued signal: both forms estimate the same thing
            assert abs(R[0, ia, im] - expect) < band, (a, m)
            assert abs(R[1, ia, im] - expect) < band, (a, m)


def _gmsk_case(T, bt=0.3, sps=8, f0=0.05, snr=10.0, seed=0xC7C1_0103):
    s = synth.carrier(synth.gmsk(T, bt=bt, sps=sps, seed=seed), f0)
    return synth.add_awgn(s, snr, seed=seed).astype(np.complex64)


def test_gmsk_cycle_frequency_locations():
    """Conventional lines at k/T; conjugate lines at 1/(2T) + k/T shifted by twice the
    carrier offset (Sec. 3 for h = 1/2; Sec. 5 on the carrier offset)."""
    sps, f0 = 8, 0.05
    T = (1 << 19) + 31
    x = _gmsk_case(T, sps=sps, f0=f0)
    lags = np.arange(0, 32, 2)
    conv_on, conv_off = [1 / sps, -1 / sps], [0.5 / sps, 0.3 / sps]
    conj_on = [2 * f0 + 0.5 / sps, 2 * f0 - 0.5 / sps]
    conj_off = [2 * f0, 0.1 + 1 / sps, 2 * f0 + 0.25 / sps]
    R, N = oracle.estimate(x, lags, conv_on + conv_off, CONV)
    r0 = oracle.r00(x, 30)
    pk = np.abs(R[0]).max(axis=1) / r0
    noise = 1.0 / math.sqrt(N)
    assert pk[0] > 3 * pk[2] and pk[0] > 3 * pk[3] and pk[0] > 10 * noise
    assert pk[1] > 3 * pk[2] and pk[1] > 10 * noise
    R, _ = oracle.estimate(x, lags, conj_on + conj_off, CONJ)
    pk = np.abs(R[0]).max(axis=1) / r0
    assert np.all(pk[:2] > 0.1) and np.all(pk[2:] < 10 * noise)


def test_cpm_not_half_integer_index_is_proper():
    """CPM with h = 0.7 has no conjugate cycle frequencies (Sec. 3)."""
    sps, T = 8, (1 << 16) + 15
    s = synth.cpm(T, h=0.7, sps=sps, pulse=synth.gaussian_freq_pulse(0.3, sps), seed=0xC7C1_0104)
    x = s.astype(np.complex64)
    al = np.array([0.0, 0.5 / sps, 1 / sps, 1.5 / sps, 0.7 / sps, 0.35 / sps])
    R, N = oracle.estimate(x, np.arange(0, 16, 3), al, CONJ)
    G, _ = oracle.estimate(synth.gmsk(T, bt=0.3, sps=sps, seed=0xC7C1_0104), np.arange(0, 16, 3), al, CONJ)
    assert np.abs(R).max() < 0.1 * np.abs(G).max()
    assert np.abs(R).max() < 20.0 / math.sqrt(N)


def test_table1_experiment_replica():
    """Synthetic replica of experiments 1 and 2 with the Table 1 parameters (Sec. 5):
    the cyclic ACF line at 1/T and the cyclic CCF line at 1/(2T) are present, and absent
    at nearby non-cycle frequencies, on windows of win_len samples."""
    with open(os.path.join(GOLD, "table1_gmsk.json")) as f:
        t1 = json.load(f)
    sps = t1["samples_per_symbol"]
    assert t1["sample_rate_hz"] == sps * t1["baud_rate"]
    a_exp1 = t1["baud_rate"] / t1["sample_rate_hz"]
    b_exp2 = 0.5 * t1["baud_rate"] / t1["sample_rate_hz"]
    assert a_exp1 == t1["experiment_1_alpha_norm"] and b_exp2 == t1["experiment_2_beta_norm"]
    N, M = t1["win_len"], t1["max_lag"]
    # 64 consecutive windows of win_len samples in one record: the weak conventional GMSK
    # feature needs the longer average to stand clear of the estimator's own noise.  The
    # conventional feature lives at lags within three symbols; the CCF one extends further.
    x = synth.gmsk(64 * N + M, bt=t1["BT"], sps=sps, seed=0xC7C1_0105).astype(np.complex64)
    Rc, _ = oracle.estimate(x, np.arange(0, 3 * sps + 1, 2), [a_exp1, 0.75 * a_exp1, 0.5 * a_exp1], CONV)
    Rj, _ = oracle.estimate(x, np.arange(0, M + 1, 4), [b_exp2, 1.5 * b_exp2, 0.5 * b_exp2], CONJ)
    pc = np.abs(Rc[0]).max(axis=1)
    pj = np.abs(Rj[0]).max(axis=1)
    assert pc[0] > 4 * pc[1] and pc[0] > 4 * pc[2]
    assert pj[0] > 10 * pj[1] and pj[0] > 10 * pj[2]
