"""Eq. (impl-corr) in full on the GPU: signed lags (window starting M^- samples in) and two
inputs (cyc_create_xy / cyc_push_xy), against the oracle's estimate_xy, element by element,
in every precision.  Error metric: max |R_gpu - R_oracle| over sqrt(mean|x|^2 mean|y|^2)
on the committed range (R^0(0) when y = x)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "fp16": 1e-2}
PRECS = ["fp32", "bf16x3", "fp16"]


def norm(x, y, lags):
    lo, hi = min(0, int(np.min(lags))), max(0, int(np.max(lags)))
    return oracle.r00_xy(x, y, -lo, hi)


def run(cyc, x, y, lags, alphas, precision, chunks=None, forms=3, n0=0):
    import torch
    cross = y is not None
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda() if cross else None
    with cyc.Stream(lags, alphas, forms, precision=precision, n0=n0, cross=cross) as s:
        pos = 0
        for c in (chunks or [x.size]):
            if cross:
                s.push(xt[2 * pos:2 * (pos + c)], y=yt[2 * pos:2 * (pos + c)])
            else:
                s.push(xt[2 * pos:2 * (pos + c)])
            pos += c
        R, neff = s.read()
    return R, neff


def pair_signal(T, seed, delay=5, f=0.07):
    """x white; y[n] = x[n + delay] exp(j 2 pi f n) plus noise: a cross line (CONV) at
    a = -f and lag m = delay, since x[n + delay] conj(y[n]) ~ |x[n + delay]|^2 exp(-j 2 pi f n)."""
    s = synth.white(T + delay, seed=seed)
    n = np.arange(T)
    x = s[:T]
    y = s[delay:T + delay] * np.exp(2j * np.pi * f * n) + 0.3 * synth.white(T, seed=seed + 1)
    return x.astype(np.complex64), y.astype(np.complex64)


@pytest.mark.parametrize("precision", PRECS)
def test_signed_lags_one_input(cyc, precision):
    x = synth.white(9001, seed=140).astype(np.complex64)
    lags = np.array([-40, -7, -1, 0, 3, 17, 100])
    alphas = np.random.default_rng(40).uniform(-0.5, 0.5, 37)
    R, neff = run(cyc, x, None, lags, alphas, precision, chunks=[3000, 6001])
    Ro, no = oracle.estimate_xy(x, None, lags, alphas)
    assert neff == no == 9001 - 140
    assert np.max(np.abs(R - Ro)) / norm(x, None, lags) < TOL[precision]


@pytest.mark.parametrize("precision", PRECS)
def test_cross_forms(cyc, precision):
    x, y = pair_signal(12007, seed=141)
    lags = np.arange(-20, 21)
    alphas = np.concatenate([[0.0, -0.07, 0.07], np.random.default_rng(41).uniform(-0.5, 0.5, 47)])
    R, neff = run(cyc, x, y, lags, alphas, precision, chunks=[5000, 7007])
    Ro, no = oracle.estimate_xy(x, y, lags, alphas)
    assert neff == no == 12007 - 40
    assert np.max(np.abs(R - Ro)) / norm(x, y, lags) < TOL[precision]
    # the planted line: CONV, a = -f, lag m = 5 (x[n+5] is the y-carrier's source sample)
    assert abs(Ro[0, 1, 25]) > 0.5 * norm(x, y, lags)


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_cross_tensor_core_tiles(cyc, precision):
    """Wide items (128 lags x 2 forms), an odd number of cycle-frequency tiles (pairs with an
    empty partner), several staged blocks per item, and a narrow second column range."""
    x, y = pair_signal(20011, seed=142)
    for lags in (np.arange(-64, 64), np.arange(-70, 90)):
        alphas = np.random.default_rng(42).uniform(-0.5, 0.5, 300)
        R, neff = run(cyc, x, y, lags, alphas, precision, chunks=[7777, 12234])
        Ro, no = oracle.estimate_xy(x, y, lags, alphas)
        assert neff == no
        assert np.max(np.abs(R - Ro)) / norm(x, y, lags) < TOL[precision], lags.min()


@pytest.mark.parametrize("precision", PRECS)
def test_cross_chunk_split_and_large_start(cyc, precision):
    x, y = pair_signal(3001, seed=143)
    lags = np.array([-9, 0, 4, 12])
    alphas = np.array([0.0, 0.25, -0.07, 0.333])
    n0 = (1 << 40) + 12345
    Ro, _ = oracle.estimate_xy(x, y, lags, alphas, n0=n0)
    for chunks in ([3001], [1, 5, 20, 21, 800, 2154], [21] * 142 + [19]):
        assert sum(chunks) == 3001
        R, _ = run(cyc, x, y, lags, alphas, precision, chunks=chunks, n0=n0)
        assert np.max(np.abs(R - Ro)) / norm(x, y, lags) < TOL[precision], chunks[:3]


def test_cross_save_load_and_errors(cyc):
    import torch
    x, y = pair_signal(4000, seed=144)
    lags, alphas = np.array([-3, 0, 6]), np.array([0.0, 0.1])
    Ro, _ = oracle.estimate_xy(x, y, lags, alphas)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda()
    with cyc.Stream(lags, alphas, 3, cross=True) as s1, cyc.Stream(lags, alphas, 3, cross=True) as s2:
        s1.push(xt[:2 * 1500], y=yt[:2 * 1500])
        s2.load(s1.save())
        s2.push(xt[2 * 1500:], y=yt[2 * 1500:])
        R, _ = s2.read()
        assert np.max(np.abs(R - Ro)) / norm(x, y, lags) < 1e-5
        with pytest.raises(cyc.CycError) as e:
            cyc.cyc_push(s1.h, xt)
        assert e.value.code == cyc.CYC_EINVAL
    with cyc.Stream(lags, alphas, 3) as s:
        with pytest.raises(cyc.CycError) as e:
            cyc.cyc_push_xy(s.h, xt, yt)
        assert e.value.code == cyc.CYC_EINVAL
        with cyc.Stream([0, 1], alphas, 3) as other:
            with pytest.raises(cyc.CycError):
                other.load(s.save())
    with pytest.raises(cyc.CycError) as e:
        cyc.Stream([-2000, 1000], [0.1], 3, precision="bf16x3")
    assert e.value.code == cyc.CYC_ENOTSUP
    with pytest.raises(cyc.CycError) as e:
        cyc.Stream([-(1 << 20), 1 << 20], [0.1], 3)
    assert e.value.code == cyc.CYC_EINVAL
