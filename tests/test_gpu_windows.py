"""The block's windowed output on the GPU (cyc_create_window / cyc_read_windows) against the
oracle's windows: Eq. (impl-corr) at window starts k * hop with the window-local phase, one
input or two, signed lags, every precision, pushes that do not line up with hops.  Error
metric: max over a window's entries of |R_gpu - R_oracle| over sqrt(mean|x|^2 mean|y|^2) of
the whole signal."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "fp16": 1e-2}


def run_windows(cyc, x, y, lags, alphas, N, hop, precision, chunks, cap=8):
    """Push the chunks, reading windows whenever the ring is full (a chunk must not complete
    more than `cap` windows by itself); all windows, in order."""
    import torch
    cross = y is not None
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda() if cross else None
    got, ks = [], []
    with cyc.Stream(lags, alphas, 3, precision=precision, cross=cross, window=(N, hop, cap)) as s:
        pos = 0
        for c in chunks:
            sl = slice(2 * pos, 2 * (pos + c))
            while True:
                try:
                    s.push(xt[sl], y=yt[sl] if cross else None)
                    break
                except cyc.CycError as e:
                    assert e.code == cyc.CYC_EAGAIN
                    W, k0 = s.read_windows(cap)
                    assert W.shape[0] > 0
                    got.append(W.copy())
                    ks.append(k0)
            pos += c
        W, k0 = s.read_windows(1 << 16)
        got.append(W.copy())
        ks.append(k0)
        R, neff = s.read()
    k = 0
    for W, k0 in zip(got, ks):
        assert k0 == k
        k += W.shape[0]
    return np.concatenate(got), R, neff


def check(W, Wo, x, y, lags, tol):
    assert W.shape == Wo.shape, (W.shape, Wo.shape)
    lo, hi = min(0, int(np.min(lags))), max(0, int(np.max(lags)))
    nrm = oracle.r00_xy(x, y, 0, 0)
    err = np.max(np.abs(W - Wo)) / nrm
    assert err < tol, err


def ragged(T, seed):
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, T), size=9, replace=False))
    return np.diff(np.concatenate([[0], cuts, [T]]))


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16"])
def test_windows_one_input_signed_lags(cyc, precision):
    T, N, hop = 5000, 256, 64
    x = synth.white(T, seed=160).astype(np.complex64)
    lags = np.array([-6, -1, 0, 2, 5, 9])
    alphas = np.concatenate([[0.0], np.random.default_rng(60).uniform(-0.5, 0.5, 19)])
    W, R, neff = run_windows(cyc, x, None, lags, alphas, N, hop, precision, ragged(T, 61), cap=128)
    Wo = oracle.windows(x, None, lags, alphas, N, hop)
    check(W, Wo, x, None, lags, TOL[precision])
    Ro, no = oracle.estimate_xy(x, None, lags, alphas)          # the running sums are unchanged
    assert neff == no
    assert np.max(np.abs(R - Ro)) / oracle.r00_xy(x, None, 6, 9) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_windows_two_inputs(cyc, precision):
    T, N, hop = 4000, 512, 128
    x = synth.white(T, seed=162).astype(np.complex64)
    y = (np.roll(x, 3) * np.exp(2j * np.pi * 0.05 * np.arange(T)) + 0.3 * synth.white(T, seed=163)).astype(np.complex64)
    lags = np.arange(-4, 5)
    alphas = np.concatenate([[-0.05, 0.0], np.random.default_rng(62).uniform(-0.5, 0.5, 10)])
    W, _, _ = run_windows(cyc, x, y, lags, alphas, N, hop, precision, ragged(T, 63), cap=64)
    Wo = oracle.windows(x, y, lags, alphas, N, hop)
    check(W, Wo, x, y, lags, TOL[precision])


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_windows_tensor_core_tiles(cyc, precision):
    """Wide items (lags -64..63, both forms), two cycle-frequency tiles, several hops per pass."""
    T, N, hop = 12000, 2048, 512
    x = synth.white(T, seed=164).astype(np.complex64)
    lags = np.arange(-64, 64)
    alphas = np.random.default_rng(64).uniform(-0.5, 0.5, 129)
    W, _, _ = run_windows(cyc, x, None, lags, alphas, N, hop, precision, [3001, 4999, 4000], cap=32)
    Wo = oracle.windows(x, None, lags, alphas, N, hop)
    check(W, Wo, x, None, lags, TOL[precision])


def test_window_ring_backpressure_and_reset(cyc):
    import torch
    T, N, hop = 2000, 128, 32
    x = synth.white(T, seed=165).astype(np.complex64)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    lags, alphas = np.array([0, 3]), np.array([0.0, 0.21])
    Wo = oracle.windows(x, None, lags, alphas, N, hop)
    with cyc.Stream(lags, alphas, 3, window=(N, hop, 2)) as s:
        s.push(xt[:2 * (N + 3 + hop)])             # windows 0 and 1 complete: the ring is full
        with pytest.raises(cyc.CycError) as e:
            s.push(xt[2 * (N + 3 + hop):2 * (N + 3 + 2 * hop)])
        assert e.value.code == cyc.CYC_EAGAIN
        W, k0 = s.read_windows(1)
        assert k0 == 0 and W.shape[0] == 1
        s.push(xt[2 * (N + 3 + hop):2 * (N + 3 + 2 * hop)])
        W2, k1 = s.read_windows(8)
        assert k1 == 1 and W2.shape[0] == 2
        assert np.max(np.abs(np.concatenate([W, W2]) - Wo[:3])) < 1e-5
        s.reset()
        s.push(xt[:2 * (N + 3)])
        W3, k3 = s.read_windows(8)
        assert k3 == 0 and W3.shape[0] == 1 and np.max(np.abs(W3[0] - Wo[0])) < 1e-5
        with pytest.raises(cyc.CycError) as e:
            s.save()
        assert e.value.code == cyc.CYC_ENOTSUP
    with pytest.raises(cyc.CycError):
        cyc.Stream(lags, alphas, 3, window=(100, 32, 4))     # win_len not a multiple of hop
    with cyc.Stream(lags, alphas, 3) as s:
        with pytest.raises(cyc.CycError) as e:
            s.read_windows(1)
        assert e.value.code == cyc.CYC_EINVAL


def test_windows_long_stream_no_drift(cyc):
    """16 384 hops through the add-one/drop-one window update: the last windows equal the
    oracle's estimate over just their own samples (the window-local phase makes a window
    depend on nothing else), so error carried along the stream would show here."""
    import torch
    T, N, hop, C = 1 << 20, 4096, 64, 1 << 16
    lags = np.arange(8)
    alphas = np.concatenate([[0.0], np.random.default_rng(70).uniform(-0.5, 0.5, 19)])
    x = synth.white(T, seed=170).astype(np.complex64)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    cap = C // hop + 1
    last, k_last = None, None
    with cyc.Stream(lags, alphas, 3, precision="fp32", max_chunk=C, window=(N, hop, cap)) as s:
        for c in range(T // C):
            s.push(xt[2 * c * C:2 * (c + 1) * C])
            W, k0 = s.read_windows(cap)
            if W.shape[0]:
                last, k_last = W.copy(), k0
    M = int(lags.max())
    nrm = oracle.r00_xy(x, None, 0, 0)
    for i in (0, last.shape[0] // 2, last.shape[0] - 1):
        k = k_last + i
        Wo = oracle.windows(x[k * hop:k * hop + N + M], None, lags, alphas, N, hop)[0]
        assert np.max(np.abs(last[i] - Wo)) / nrm < 1e-5, (k, np.max(np.abs(last[i] - Wo)) / nrm)
    assert k_last + last.shape[0] - 1 == (T - M - N) // hop


@pytest.mark.parametrize("hop,nalpha,N", [(1, 6, 64), (5, 40, 125), (3, 12, 96)])
def test_windows_at_short_hops(cyc, hop, nalpha, N):
    """Hops below 16 samples, down to hop = 1 (an estimate per input sample, the block's own
    output rate), on the FP32 path (few cycle frequencies: register sums; more: the tiled
    kernel): every window against the oracle; tensor-core precisions refuse such hops."""
    T = 3000
    x = synth.white(T, seed=190).astype(np.complex64)
    lags = np.array([-2, 0, 1, 4, 7])
    alphas = np.random.default_rng(191).uniform(-0.5, 0.5, nalpha)
    W, R, neff = run_windows(cyc, x, None, lags, alphas, N, hop, "fp32", ragged(T, 192), cap=T)
    Wo = oracle.windows(x, None, lags, alphas, N, hop)
    check(W, Wo, x, None, lags, TOL["fp32"])
    Ro, no = oracle.estimate_xy(x, None, lags, alphas)
    assert neff == no and np.max(np.abs(R - Ro)) / oracle.r00_xy(x, None, 2, 7) < TOL["fp32"]
    with pytest.raises(cyc.CycError) as e:
        cyc.Stream(lags, alphas, 3, precision="bf16x3", window=(N, hop, 4))
    assert e.value.code == cyc.CYC_EINVAL
