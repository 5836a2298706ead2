"""Pins of the reduced-precision operand emulation (CPU): bf16 / fp16 rounding on values
whose rounding is fixed by the formats, the split's reconstruction and product error bounds,
and exact agreement with the FP64 oracle when every operand is representable."""
import numpy as np

import oracle
from oracle import split


def test_bf16_round_to_nearest_even_cases():
    u = 2.0 ** -7                                       # bf16 spacing just above 1
    cases = {1.0: 1.0, 1 + u / 2: 1.0, 1 + 1.5 * u: 1 + 2 * u, 1 + 0.75 * u: 1 + u,
             -(1 + u / 2): -1.0, 3.0: 3.0, 2.0 ** -130: 2.0 ** -130, 0.0: 0.0}
    for v, want in cases.items():
        assert split.bf16_rn(np.array([v]))[0] == want, v


def test_fp16_round_to_nearest_even_cases():
    u = 2.0 ** -10
    for v, want in {1 + u / 2: 1.0, 1 + 1.5 * u: 1 + 2 * u, 65504.0: 65504.0}.items():
        assert split.fp16_rn(np.array([v]))[0] == want


def test_split_reconstruction_and_product_bounds():
    rng = np.random.default_rng(0)
    a = rng.normal(size=10000).astype(np.float32).astype(np.float64)
    b = rng.normal(size=10000).astype(np.float32).astype(np.float64)
    ah, al = split.split_bf16(a)
    bh, bl = split.split_bf16(b)
    assert np.all(np.abs(a - ah) <= 2.0 ** -8 * np.abs(a))            # hi: 8 significant bits
    assert np.all(np.abs(a - ah - al) <= 2.0 ** -16 * np.abs(a))      # hi + lo: 16 bits
    err = np.abs(ah * bh + ah * bl + al * bh - a * b)
    assert np.all(err <= 2.0 ** -14 * np.abs(a * b))
    assert np.median(err / np.abs(a * b)) > 2.0 ** -24                # the split does lose bits


def test_exact_operands_reproduce_the_oracle():
    """x in {+-1, +-1/2, +-j}: every lag product is exact in bf16 and fp16; with a = 0 and
    a = 1/2 every weight is +-1, so both emulations equal the FP64 oracle exactly."""
    rng = np.random.default_rng(1)
    x = rng.choice(np.array([1, -1, 0.5, -0.5, 1j, -1j]), size=64)
    lags, alphas = [0, 1, 5], [0.0, 0.5]
    Ro, N = oracle.estimate(x, lags, alphas)
    for prec in ("bf16x3", "fp16"):
        Re, Ne = split.estimate_rounded(x, lags, alphas, precision=prec)
        assert Ne == N
        assert np.max(np.abs(Re - Ro)) < 1e-15, prec
