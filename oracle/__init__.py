"""FP64 CPU oracle for the cyclic correlation estimator -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product path (``paper_2405_16911_gb300``) never imports it and
shares no code with it; the two meet only through the seeded generators in ``synth``.

``estimate`` follows paper Sec. 4 Eq. (impl-corr) with x = y, m >= 0, absolute sample
index n (origin at the first pushed sample) and normalisation by the number of terms
N_eff = T - max(lags), as written out in ``cyc_oracle.c``; ``estimate_xy`` is the same
equation in full (two inputs, signed lags, N_eff = T - M^- - M^+).  Its pins (closed forms,
DFT special cases, brute force, invariants, statistics) live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cyc_oracle.c")
_LIB = os.path.join(_HERE, "libcyc_oracle.so")
_lock = threading.Lock()
_lib = None

CONV, CONJ = 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, dp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
            lib.cyco_estimate.argtypes = [dp, i64, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                          i64, ctypes.c_int, dp, ctypes.POINTER(i64)]
            lib.cyco_estimate.restype = ctypes.c_int
            lib.cyco_entries.argtypes = [dp, i64, i32, ctypes.c_int, dp, dp, dp, i64, ctypes.c_int,
                                         dp, ctypes.POINTER(i64)]
            lib.cyco_entries.restype = ctypes.c_int
            lib.cyco_r00.argtypes = [dp, i64, i32]
            lib.cyco_r00.restype = ctypes.c_double
            lib.cyco_estimate_xy.argtypes = [dp, dp, i64, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                             i64, ctypes.c_int, dp, ctypes.POINTER(i64)]
            lib.cyco_estimate_xy.restype = ctypes.c_int
            lib.cyco_r00_xy.argtypes = [dp, dp, i64, i32, i32]
            lib.cyco_r00_xy.restype = ctypes.c_double
            lib.cyco_windows.argtypes = [dp, dp, i64, dp, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, i64, i64,
                                         i64, ctypes.c_int, dp, ctypes.POINTER(i64)]
            lib.cyco_windows.restype = ctypes.c_int
            lib.cyco_max_threads.argtypes = []
            lib.cyco_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().cyco_max_threads())


def _as_x(x) -> np.ndarray:
    x = np.ascontiguousarray(np.asarray(x).astype(np.complex128))
    return x.view(np.float64)


def _forms_list(forms: int):
    return [f for f in (CONV, CONJ) if forms & f]


def estimate(x, lags, alphas, forms: int = CONV | CONJ, n0: int = 0, threads: int = 0):
    """R as a complex128 array [F][len(alphas)][len(lags)] and N_eff.

    x is widened to complex128 as given (pass the complex64 workload to check a GPU result).
    Raises ValueError on bad arguments; returns (None, 0) when N_eff == 0.
    """
    lib = _load()
    xf = _as_x(x)
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    F = len(_forms_list(forms))
    out = np.zeros((F, alphas.size, lags.size, 2), dtype=np.float64)
    neff = ctypes.c_int64(0)
    rc = lib.cyco_estimate(xf.ctypes.data, xf.size // 2, lags.ctypes.data, lags.size,
                           alphas.ctypes.data, alphas.size, forms, int(n0),
                           threads or max_threads(), out.ctypes.data, ctypes.byref(neff))
    if rc == -2:
        return None, 0
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out[..., 0] + 1j * out[..., 1], int(neff.value)


def entries(x, M: int, form, alphas, lag, n0: int = 0, threads: int = 0):
    """Selected entries (form[i], alphas[i], lag[i]) with N_eff = T - M; complex128 [nent]."""
    lib = _load()
    xf = _as_x(x)
    form = np.ascontiguousarray(np.asarray(form, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    lag = np.ascontiguousarray(np.asarray(lag, dtype=np.int32))
    out = np.zeros((form.size, 2), dtype=np.float64)
    neff = ctypes.c_int64(0)
    rc = lib.cyco_entries(xf.ctypes.data, xf.size // 2, int(M), form.size, form.ctypes.data,
                          alphas.ctypes.data, lag.ctypes.data, int(n0), threads or max_threads(),
                          out.ctypes.data, ctypes.byref(neff))
    if rc == -2:
        return None, 0
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out[:, 0] + 1j * out[:, 1], int(neff.value)


def r00(x, M: int) -> float:
    """R^0(0) over the first T - M samples: the normaliser of every parity error."""
    xf = _as_x(x)
    return float(_load().cyco_r00(xf.ctypes.data, xf.size // 2, int(M)))


def estimate_xy(x, y, lags, alphas, forms: int = CONV | CONJ, n0: int = 0, threads: int = 0):
    """Eq. (impl-corr) with two inputs (y None: y = x) and signed lags: R complex128
    [F][len(alphas)][len(lags)] and N_eff = T - M^- - M^+ (see cyc_oracle.c)."""
    lib = _load()
    xf = _as_x(x)
    yf = None if y is None else _as_x(y)
    if yf is not None and yf.size != xf.size:
        raise ValueError("oracle: x and y differ in length")
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    F = len(_forms_list(forms))
    out = np.zeros((F, alphas.size, lags.size, 2), dtype=np.float64)
    neff = ctypes.c_int64(0)
    rc = lib.cyco_estimate_xy(xf.ctypes.data, None if yf is None else yf.ctypes.data, xf.size // 2,
                              lags.ctypes.data, lags.size, alphas.ctypes.data, alphas.size, forms, int(n0),
                              threads or max_threads(), out.ctypes.data, ctypes.byref(neff))
    if rc == -2:
        return None, 0
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out[..., 0] + 1j * out[..., 1], int(neff.value)


def r00_xy(x, y, Mneg: int, Mpos: int) -> float:
    """sqrt(mean|x|^2 mean|y|^2) over the committed range [M^-, T - M^+): the normaliser of
    cross parity errors (R^0(0) there when y is None)."""
    xf = _as_x(x)
    yf = None if y is None else _as_x(y)
    return float(_load().cyco_r00_xy(xf.ctypes.data, None if yf is None else yf.ctypes.data, xf.size // 2,
                                     int(Mneg), int(Mpos)))


def windows(x, y, lags, alphas, win_len: int, hop: int, forms: int = CONV | CONJ, max_win: int = 1 << 20,
            threads: int = 0):
    """The block's windowed output, Eq. (impl-corr) at window starts n0 = k * hop with the
    window-local phase: complex128 [nwin][F][len(alphas)][len(lags)] (see cyc_oracle.c)."""
    lib = _load()
    xf = _as_x(x)
    yf = None if y is None else _as_x(y)
    if yf is not None and yf.size != xf.size:
        raise ValueError("oracle: x and y differ in length")
    lags = np.ascontiguousarray(np.asarray(lags, dtype=np.int32))
    alphas = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    F = len(_forms_list(forms))
    T = xf.size // 2
    span = max(0, -int(lags.min())) + max(0, int(lags.max())) + int(win_len)
    nmax = max(0, (T - span) // int(hop) + 1) if T >= span else 0
    nmax = min(nmax, int(max_win))
    out = np.zeros((max(nmax, 1), F, alphas.size, lags.size, 2), dtype=np.float64)
    nw = ctypes.c_int64(0)
    rc = lib.cyco_windows(xf.ctypes.data, None if yf is None else yf.ctypes.data, T, lags.ctypes.data, lags.size,
                          alphas.ctypes.data, alphas.size, forms, int(win_len), int(hop), nmax,
                          threads or max_threads(), out.ctypes.data, ctypes.byref(nw))
    if rc != 0:
        raise ValueError("oracle: bad arguments")
    return out[:nmax, ..., 0] + 1j * out[:nmax, ..., 1]


def lag_window(lags, taper: int) -> np.ndarray:
    """Lag weights: taper 0 rectangular (1), taper 1 Hann centred on m = 0,
    w(m) = 0.5 + 0.5 cos(pi m / (Mmax + 1)) with Mmax = max |m|."""
    lags = np.asarray(lags, dtype=np.float64)
    if taper == 0:
        return np.ones_like(lags)
    mmax = np.max(np.abs(lags))
    return 0.5 + 0.5 * np.cos(np.pi * lags / (mmax + 1.0))


def spectrum(R, lags, Q: int, taper: int = 0) -> np.ndarray:
    """Cyclic spectrum of an estimate R [F][A][L] over its lags (cyclic correlogram):
    S[f][a][q] = sum_l w(m_l) R[f][a][l] exp(-j 2 pi f_q m_l), f_q = -1/2 + q/Q.
    Written as the plain double sum (FP64); complex128 [F][A][Q]."""
    R = np.asarray(R, dtype=np.complex128)
    lags = np.asarray(lags)
    w = lag_window(lags, taper)
    S = np.zeros(R.shape[:2] + (int(Q),), dtype=np.complex128)
    for q in range(int(Q)):
        fq = -0.5 + q / Q
        e = w * np.exp(-2j * np.pi * np.mod(fq * lags, 1.0))
        S[..., q] = np.tensordot(R, e, axes=([2], [0]))
    return S
