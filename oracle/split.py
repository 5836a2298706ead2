"""Reduced-precision operand arithmetic of the tensor-core projection, emulated in FP64 --
TEST INFRASTRUCTURE (only tests may import it).

The tensor-core path forms the weights W = exp(-j 2 pi a n) and the lag products
P = x[n+m] c(x[n]) in FP32, rounds them to 16-bit operands and accumulates in FP32:

* FP16 single pass: W16 = fp16_rn(W), P16 = fp16_rn(P); term W16 * P16.
* BF16x3 split (the 3-term BF16 split): v = hi + lo with
  hi = bf16_rn(v), lo = bf16_rn(v - hi); term hi_W hi_P + hi_W lo_P + lo_W hi_P (the
  lo_W lo_P product dropped).

Here the rounding follows those definitions bit for bit (bf16_rn: round-to-nearest-even of an
FP32 value to its top 16 bits) and every product and sum is exact FP64, so
``estimate_rounded`` shows the operands' own rounding error without the accumulation's.
Applied to complex values, each of the real and imaginary parts is rounded.
"""
from __future__ import annotations

import numpy as np


def bf16_rn(v) -> np.ndarray:
    """Round FP32 values (given as any float array) to bfloat16, nearest-even; returned as
    float64.  FP32 bits b -> (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000."""
    f = np.asarray(v, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def fp16_rn(v) -> np.ndarray:
    """Round FP32 values to IEEE binary16, nearest-even (numpy's conversion); as float64."""
    return np.asarray(v, dtype=np.float32).astype(np.float16).astype(np.float64)


def split_bf16(v):
    """(hi, lo) of FP32 values: hi = bf16_rn(v), lo = bf16_rn(v - hi) (v - hi is exact in FP32)."""
    f = np.asarray(v, dtype=np.float32).astype(np.float64)
    hi = bf16_rn(f)
    lo = bf16_rn((f - hi).astype(np.float32))
    return hi, lo


def _cround(z, fn):
    z = np.asarray(z, dtype=np.complex128)
    return fn(z.real.astype(np.float32)) + 1j * fn(z.imag.astype(np.float32))


def estimate_rounded(x, lags, alphas, forms: int = 3, precision: str = "bf16x3"):
    """The estimator of Sec. 4 Eq. (impl-corr) (x = y, lags >= 0, n0 = 0) with the operands
    rounded as the tensor-core path rounds them: [F][A][L] complex128, N_eff.

    W and P are formed in FP64, rounded to FP32 (the kernel forms them in FP32), then to the
    16-bit operands; products and sums are exact FP64.  The complex product W * P is written
    as its real parts, each one a sum of real operand products as the two real GEMMs form it."""
    x = np.asarray(x, dtype=np.complex128)
    lags = np.asarray(lags)
    M = int(lags.max())
    N = x.size - M
    n = np.arange(N)
    fl = [f for f in (1, 2) if forms & f]
    out = np.zeros((len(fl), len(alphas), len(lags)), dtype=np.complex128)
    for ia, a in enumerate(alphas):
        ph = np.mod(float(a) * n, 1.0)
        W = np.exp(-2j * np.pi * ph)
        Wr, Wi = W.real.astype(np.float32), W.imag.astype(np.float32)
        for fi, f in enumerate(fl):
            for im, m in enumerate(lags):
                c = np.conj(x[:N]) if f == 1 else x[:N]
                P = x[m:m + N] * c
                Pr, Pi = P.real.astype(np.float32), P.imag.astype(np.float32)
                if precision == "fp16":
                    wr, wi, pr, pi = fp16_rn(Wr), fp16_rn(Wi), fp16_rn(Pr), fp16_rn(Pi)
                    re = wr * pr - wi * pi
                    imv = wr * pi + wi * pr
                else:
                    (wrh, wrl), (wih, wil) = split_bf16(Wr), split_bf16(Wi)
                    (prh, prl), (pih, pil) = split_bf16(Pr), split_bf16(Pi)

                    def mul3(ah, al, bh, bl):
                        return ah * bh + ah * bl + al * bh

                    re = mul3(wrh, wrl, prh, prl) - mul3(wih, wil, pih, pil)
                    imv = mul3(wrh, wrl, pih, pil) + mul3(wih, wil, prh, prl)
                out[fi, ia, im] = (re.sum() + 1j * imv.sum()) / N
    return out, N
