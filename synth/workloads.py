"""Seeded synthetic stand-ins for the paper's over-the-air GMSK captures (Sec. 5).

The paper measured on USRP captures that are not available; these generators give signals
of the same kind (GMSK, Sec. 3; Table 1 parameters) with the shapes of the five workload
configurations.  Seeds are 0xC7C10000 + configuration index (+ stream id for serving).
Only inputs are built here (signals, lag lists, cycle-frequency grids): no estimator
arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import add_awgn, carrier, gmsk, rrc_psk, uniform01

SEED_BASE = 0xC7C1_0000


def gmsk_stream(T: int, *, bt: float, sps: int, f0: float, snr_db: float, seed: int) -> np.ndarray:
    """GMSK (h = 1/2, L = 4) with carrier offset f0 and AWGN, returned as complex64."""
    x = carrier(gmsk(T, bt=bt, sps=sps, seed=seed), f0)
    return add_awgn(x, snr_db, seed=seed).astype(np.complex64)


def config0(T: int = 65536):
    """Plain estimator, one chunk: GMSK BT 0.3, 8 sps, offset 0.05, 10 dB; lags 0..31;
    64 cycle frequencies per form: k/8 (CONV) and 0.1 + k/8 (CONJ), k = -32..31."""
    seed = SEED_BASE + 0
    k = np.arange(-32, 32)
    return dict(
        name="cfg0-gmsk-65536-lags32-a64",
        x=gmsk_stream(T, bt=0.3, sps=8, f0=0.05, snr_db=10.0, seed=seed),
        lags=np.arange(32, dtype=np.int32),
        alphas_conv=k / 8.0,
        alphas_conj=0.1 + k / 8.0,
        chunk=T,
    )


def config1(T: int = 1 << 26, replica: int = 0):
    """Streaming: GMSK as config 0, 2^26 samples pushed in 2^16-sample chunks, lags 0..127,
    1024 cycle frequencies -0.5 + k/1024, both forms.  `replica` > 0 draws an independent
    stream of the same kind (one per process when several GPUs each run their own)."""
    seed = SEED_BASE + 1 + 0x10000 * replica
    return dict(
        name="cfg1-gmsk-stream-2^26-chunk2^16-lags128-a1024-both",
        x=gmsk_stream(T, bt=0.3, sps=8, f0=0.05, snr_db=10.0, seed=seed),
        lags=np.arange(128, dtype=np.int32),
        alphas=-0.5 + np.arange(1024) / 1024.0,
        chunk=1 << 16,
    )


def config2(T: int = 1 << 20):
    """Precision: one block of 2^20 GMSK samples, BT 0.5, 4 sps, offset U(-0.25, 0.25),
    0 dB; lags 0..255; 4096 cycle frequencies -0.5 + k/4096, both forms."""
    seed = SEED_BASE + 2
    f0 = float(uniform01(seed, 9, 0, 1)[0]) * 0.5 - 0.25
    return dict(
        name="cfg2-gmsk-block-2^20-lags256-a4096-both",
        x=gmsk_stream(T, bt=0.5, sps=4, f0=f0, snr_db=0.0, seed=seed),
        f0=f0,
        lags=np.arange(256, dtype=np.int32),
        alphas=-0.5 + np.arange(4096) / 4096.0,
        chunk=T,
    )


def mix_stream_params(sid: int, seed_base: int = SEED_BASE + 3):
    """Parameters of serving stream `sid` in the config-3 mix: GMSK BT 0.3/0.5 or RRC(0.35)
    BPSK/QPSK, sps U{2..16}, offset U(-0.25, 0.25), SNR U(-5, 20) dB."""
    seed = seed_base + sid
    u = uniform01(seed, 10, 0, 4)
    kind = int(u[0] * 4)                       # 0: GMSK 0.3, 1: GMSK 0.5, 2: RRC BPSK, 3: RRC QPSK
    sps = 2 + int(u[1] * 15)
    f0 = u[2] * 0.5 - 0.25
    snr = -5.0 + 25.0 * u[3]
    return dict(kind=kind, sps=sps, f0=f0, snr_db=snr, seed=seed)


def mix_stream(sid: int, T: int, seed_base: int = SEED_BASE + 3) -> np.ndarray:
    p = mix_stream_params(sid, seed_base)
    if p["kind"] < 2:
        s = gmsk(T, bt=0.3 if p["kind"] == 0 else 0.5, sps=p["sps"], seed=p["seed"])
    else:
        s = rrc_psk(T, sps=p["sps"], beta=0.35, qpsk=p["kind"] == 3, seed=p["seed"])
    s = carrier(s, p["f0"])
    return add_awgn(s, p["snr_db"], seed=p["seed"]).astype(np.complex64)
