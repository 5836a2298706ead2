"""The seeded generators: published splitmix64 vector, block independence, pulse conditions."""
import math

import numpy as np

import synth


def test_splitmix64_published_first_output():
    # splitmix64 seeded with 0 returns 0xE220A8397B1DCDAF first (Steele et al. reference code)
    assert int(synth._mix(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF


def test_counter_streams_are_position_addressable():
    a = synth.splitmix64(7, 3, 0, 100)
    b = synth.splitmix64(7, 3, 40, 60)
    assert np.array_equal(a[40:], b)
    z = synth.normal_pairs(7, 3, 0, 20000)
    assert abs(np.mean(z.real)) < 0.05 and abs(np.var(z.real) - 1) < 0.05 and abs(np.var(z.imag) - 1) < 0.05


def test_gmsk_pulse_conditions_and_envelope():
    f = synth.gaussian_freq_pulse(0.3, 8, 4)
    assert f.size == 32 and abs(f.sum() - 0.5) < 1e-15     # condition (c)
    assert np.allclose(f, f[::-1], atol=1e-15)               # condition (b)
    x = synth.gmsk(5000, bt=0.3, sps=8, seed=1)
    assert np.allclose(np.abs(x), 1.0, atol=1e-12)           # constant envelope
    # block-size independence up to summation order
    y = synth.cpm(5000, h=0.5, sps=8, pulse=f, seed=1, block=777)
    assert np.allclose(x, y, atol=1e-9)
    # Eq. (cpm) written out directly: x[n] = exp(j 2 pi h sum_k a_k g[n - k sps]) with the
    # phase response g = running sum of f, equal to 1/2 once the pulse has passed
    g = np.cumsum(f)
    a = synth.symbols_pm1(1, 0, 0, 5000 // 8 + 1)
    n = np.arange(600)
    ph = np.zeros(n.size)
    for k in range(n.size // 8 + 1):
        d = n - 8 * k
        gk = np.where(d < 0, 0.0, np.where(d >= 32, 0.5, g[np.clip(d, 0, 31)]))
        ph += a[k] * gk
    assert np.allclose(x[:600], np.exp(2j * np.pi * 0.5 * ph), atol=1e-12)


def test_rrc_unit_power_and_blocks():
    h = synth.rrc_taps(0.35, 4)
    assert abs(np.sum(h * h) - 4) < 1e-12
    x = synth.rrc_psk(60000, sps=4, beta=0.35, qpsk=True, seed=2)
    assert abs(np.mean(np.abs(x[200:]) ** 2) - 1.0) < 0.05
    y = synth.rrc_psk(60000, sps=4, beta=0.35, qpsk=True, seed=2, block=1001)
    assert np.allclose(x, y, atol=1e-12)
