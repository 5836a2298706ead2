"""Cycle-frequency detection rule, plain numpy FP64 -- TEST INFRASTRUCTURE.

Only tests, smoke() and bench.py's baseline leg may import this module; the product path
(libcyc's cyc_detect) shares no code with it.

The paper names cycle-frequency estimation as its next step (Sec. 6) without giving a rule.
The reading used here is a constant-false-alarm (CFAR) test per form on the estimate
R [F][A][L] of a stream whose cycle frequencies form a circular grid (the order of the
stream's list, e.g. a_k = -1/2 + k/A):

    s(f, a)   = max over lags m of |R_f^a(m)|^2, with s = 0 for the conventional form at
                a = 0 (mod 1) of a one-input stream (that line is the signal's power, always
                present)
    nu(f, a)  = median of s(f, a + d) over the 2 (win - 1) offsets d = +-2 .. +-win, indices
                taken modulo A (numpy's median: the mean of the two middle values)
    ratio     = s / max(nu, tiny)
    local max = s(f, a) >= s(f, a - 1) and s(f, a) >= s(f, a + 1)
    detected  = ratio > kappa and local max

The pins are in tests/test_oracle_detect_pins.py (constructed cases for every clause, a
tone's conjugate line, GMSK line locations, white noise without false alarms).
"""
from __future__ import annotations

import numpy as np

KAPPA = 8.4
WIN = 16
TINY = 1e-300


def statistic(R, alphas=None, forms=(1, 2), exclude_conv_dc: bool = True):
    """s [F][A] = max over lags of |R|^2 (conventional a = 0 mod 1 set to 0)."""
    s = (np.abs(np.asarray(R, dtype=np.complex128)) ** 2).max(axis=-1)
    if exclude_conv_dc and alphas is not None:
        dc = np.asarray([float(a) % 1.0 == 0.0 for a in alphas])
        for fi, f in enumerate(forms):
            if f == 1:
                s[fi, dc] = 0.0
    return s


def cfar(R, alphas=None, forms=(1, 2), kappa: float = KAPPA, win: int = WIN, exclude_conv_dc: bool = True):
    """(detected [F][A] bool, ratio [F][A], local maximum [F][A] bool) of the rule above."""
    s = statistic(R, alphas, forms, exclude_conv_dc)
    F, A = s.shape
    offs = np.array([d for d in range(-win, win + 1) if abs(d) > 1])
    idx = (np.arange(A)[:, None] + offs[None, :]) % A
    nu = np.median(s[:, idx], axis=2)
    ratio = s / np.maximum(nu, TINY)
    lm = (s >= np.roll(s, 1, axis=1)) & (s >= np.roll(s, -1, axis=1))
    return (ratio > kappa) & lm, ratio, lm
