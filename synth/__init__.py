"""Seeded synthetic signal generators shared by the oracle tests, the GPU tests and the bench.

This module holds no cyclic-correlation arithmetic: it only draws random numbers and shapes
them into complex-baseband signals of the kinds the paper works with (CPM/GMSK, Sec. 3,
Eq. (cpm) and conditions (a)-(c); plus tones, white noise, rectangular BPSK and RRC PSK used
as test signals with known cyclic structure).

Randomness is counter based (splitmix64 on an index, Box-Muller for normals), so any block
of a long signal can be generated on its own and the result does not depend on how the
signal is cut into blocks, on the machine, or on the numpy version.

All generators return complex128 arrays computed in FP64.  Workloads are stored and fed to
both sides as complex64 (``.astype(np.complex64)``); the oracle then widens those same
complex64 samples back to FP64.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "splitmix64", "uniform01", "normal_pairs", "symbols_pm1",
    "cpm", "gmsk", "rect_bpsk", "rrc_psk", "rrc_taps", "tone", "white",
    "add_awgn", "carrier", "gaussian_freq_pulse",
]

_GOLD = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array, wrapping mod 2^64."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def splitmix64(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """``count`` 64-bit words of the counter-based stream (seed, stream) from index ``start``.

    Word i is mix(key + (i + 1) * golden) with key = mix(seed * golden + stream), i.e. the
    splitmix64 sequence seeded with ``key`` and read at position i.
    """
    with np.errstate(over="ignore"):
        key = _mix(np.array([(seed * 0x9E3779B97F4A7C15 + stream) % (1 << 64)], dtype=np.uint64))[0]
        idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
        return _mix(key + idx * _GOLD)


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each word."""
    w = splitmix64(seed, stream, start, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_pairs(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """``count`` complex numbers whose real and imaginary parts are independent N(0, 1)
    (Box-Muller on two uniforms per output; element i uses words 2i and 2i+1)."""
    u = uniform01(seed, stream, 2 * start, 2 * count)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * np.pi * u2) + 1j * (r * np.sin(2.0 * np.pi * u2))


def symbols_pm1(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """iid equiprobable +-1 symbols (top bit of each word)."""
    w = splitmix64(seed, stream, start, count)
    return np.where((w >> np.uint64(63)) == 1, 1.0, -1.0)


# ----------------------------------------------------------------------------------------
# CPM / GMSK (paper Sec. 3, Eq. (cpm), conditions (a)-(c) on the frequency pulse)
# ----------------------------------------------------------------------------------------

def gaussian_freq_pulse(bt: float, sps: int, L: int = 4) -> np.ndarray:
    """GMSK frequency pulse f sampled at the sample-bin centres (k + 1/2) Ts, k < L*sps.

    f(t) = [Q(c (t - T/2)) - Q(c (t + T/2))] / (2T) with c = 2 pi B / sqrt(ln 2), centred in
    [0, L T) (condition (a)), symmetric (condition (b)), and renormalised so the samples
    sum to 1/2 (condition (c), the discrete form of g(LT) = 1/2).
    """
    T = float(sps)
    c = 2.0 * math.pi * (bt / T) / math.sqrt(math.log(2.0))
    q = lambda v: 0.5 * math.erfc(v / math.sqrt(2.0))
    t = (np.arange(L * sps) + 0.5) - L * T / 2.0
    f = np.array([q(c * (ti - T / 2.0)) - q(c * (ti + T / 2.0)) for ti in t])
    return f * (0.5 / f.sum())


def cpm(T: int, *, h: float, sps: int, pulse: np.ndarray, seed: int, stream: int = 0,
        block: int = 1 << 20) -> np.ndarray:
    """Binary CPM x[n] = exp(j 2 pi h sum_k a_k q[n - k sps]) for n >= 0, with q the running
    sum of the sampled frequency pulse (phase response g), symbols a_k = +-1 from
    (seed, stream).  Generated in blocks with the phase carried across blocks."""
    Lf = pulse.size
    out = np.empty(T, dtype=np.complex128)
    phase0 = 0.0
    for s in range(0, T, block):
        e = min(T, s + block)
        k_lo = max(0, s // sps - (Lf // sps) - 1)
        k_hi = (e - 1) // sps + 1
        a = symbols_pm1(seed, stream, k_lo, k_hi - k_lo)
        u = np.zeros((k_hi - k_lo) * sps)
        u[::sps] = a
        y = np.convolve(u, pulse)                     # y[j] is the frequency at n = j + k_lo*sps
        off = s - k_lo * sps
        freq = y[off:off + (e - s)]
        ph = phase0 + 2.0 * math.pi * h * np.cumsum(freq)
        phase0 = ph[-1]
        out[s:e] = np.exp(1j * ph)
    return out


def gmsk(T: int, *, bt: float, sps: int, seed: int, stream: int = 0, L: int = 4) -> np.ndarray:
    """GMSK = binary CPM with h = 1/2 and a Gaussian frequency pulse of bandwidth B (Sec. 3)."""
    return cpm(T, h=0.5, sps=sps, pulse=gaussian_freq_pulse(bt, sps, L), seed=seed, stream=stream)


# ----------------------------------------------------------------------------------------
# Other test signals
# ----------------------------------------------------------------------------------------

def rect_bpsk(T: int, *, sps: int, seed: int, stream: int = 0) -> np.ndarray:
    """Rectangular-pulse BPSK: x[n] = a_{n // sps}, a = +-1, symbol boundaries at n = 0 mod sps."""
    a = symbols_pm1(seed, stream, 0, (T + sps - 1) // sps)
    return np.repeat(a, sps)[:T].astype(np.complex128)


def rrc_taps(beta: float, sps: int, span: int = 8) -> np.ndarray:
    """Root-raised-cosine taps over +-span symbols, scaled so that sum(h^2) = sps (the
    zero-stuffed, filtered symbol stream then has unit average power)."""
    t = np.arange(-span * sps, span * sps + 1) / float(sps)
    h = np.empty_like(t)
    for i, ti in enumerate(t):
        if abs(ti) < 1e-12:
            h[i] = 1.0 - beta + 4.0 * beta / math.pi
        elif beta > 0 and abs(abs(ti) - 1.0 / (4.0 * beta)) < 1e-12:
            h[i] = (beta / math.sqrt(2.0)) * ((1 + 2 / math.pi) * math.sin(math.pi / (4 * beta))
                                              + (1 - 2 / math.pi) * math.cos(math.pi / (4 * beta)))
        else:
            num = math.sin(math.pi * ti * (1 - beta)) + 4 * beta * ti * math.cos(math.pi * ti * (1 + beta))
            den = math.pi * ti * (1 - (4 * beta * ti) ** 2)
            h[i] = num / den
    return h * math.sqrt(sps / float(np.sum(h * h)))


def rrc_psk(T: int, *, sps: int, beta: float, qpsk: bool, seed: int, stream: int = 0,
            span: int = 8, block: int = 1 << 20) -> np.ndarray:
    """RRC-shaped BPSK (a = +-1) or QPSK (a = (+-1 +- j)/sqrt 2), iid symbols, zero-stuffed."""
    h = rrc_taps(beta, sps, span)
    half = span * sps
    out = np.empty(T, dtype=np.complex128)
    for s in range(0, T, block):
        e = min(T, s + block)
        k_lo = max(0, (s - half) // sps - 1)
        k_hi = (e + half) // sps + 1
        if qpsk:
            a = (symbols_pm1(seed, stream, 2 * k_lo, 2 * (k_hi - k_lo)).reshape(-1, 2)
                 @ np.array([1.0, 1j])) / math.sqrt(2.0)
        else:
            a = symbols_pm1(seed, stream, k_lo, k_hi - k_lo).astype(np.complex128)
        u = np.zeros((k_hi - k_lo) * sps, dtype=np.complex128)
        u[::sps] = a
        y = np.convolve(u, h)                    # y[j] is the sample at n = j + k_lo*sps - half
        off = s - k_lo * sps + half
        out[s:e] = y[off:off + (e - s)]
    return out


def tone(T: int, f0: float, n_start: int = 0) -> np.ndarray:
    """x[n] = exp(j 2 pi f0 n) for n = n_start .. n_start + T - 1 (phase reduced mod 1 in FP64)."""
    n = np.arange(n_start, n_start + T, dtype=np.float64)
    ph = np.mod(f0 * n, 1.0)
    return np.exp(2j * np.pi * ph)


def white(T: int, *, seed: int, stream: int = 0, start: int = 0) -> np.ndarray:
    """Unit-power circular white complex Gaussian noise."""
    return normal_pairs(seed, stream, start, T) / math.sqrt(2.0)


def carrier(x: np.ndarray, f0: float, n_start: int = 0) -> np.ndarray:
    """Multiply by the carrier offset exp(j 2 pi f0 n), absolute n."""
    return x * tone(x.size, f0, n_start)


def add_awgn(x: np.ndarray, snr_db: float, *, seed: int, stream: int = 1, p_signal: float = 1.0) -> np.ndarray:
    """Add circular complex white Gaussian noise of power p_signal / 10^(snr/10)."""
    sigma2 = p_signal / (10.0 ** (snr_db / 10.0))
    return x + math.sqrt(sigma2) * white(x.size, seed=seed, stream=stream)
