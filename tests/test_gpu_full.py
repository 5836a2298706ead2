"""The paper's Full mode on the GPU (cyc_create_full): every cycle frequency -1/2 + k/A by
folding the lag products modulo A and one FP64 DFT per column at read time, against the
oracle's direct estimate on the same grid, element by element (FP32 tolerance 1e-5 of
R^0(0))."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def grid(A):
    return -0.5 + np.arange(A) / A


def run_full(cyc, x, y, lags, A, chunks, n0=0, forms=3):
    import torch
    cross = y is not None
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda() if cross else None
    with cyc.Stream(lags, None, forms, n0=n0, cross=cross, full=A) as s:
        pos = 0
        for c in chunks:
            sl = slice(2 * pos, 2 * (pos + c))
            s.push(xt[sl], y=yt[sl] if cross else None)
            pos += c
        return s.read()


@pytest.mark.parametrize("A", [2, 64, 1024])
def test_full_grid_one_input(cyc, A):
    T = 10007
    x = synth.white(T, seed=170).astype(np.complex64)
    lags = np.arange(0, 21)
    n0 = (1 << 40) + 777
    R, neff = run_full(cyc, x, None, lags, A, [1, 4000, 3, 6003], n0=n0)
    Ro, no = oracle.estimate(x, lags, grid(A), n0=n0)
    assert neff == no
    assert np.max(np.abs(R - Ro)) / oracle.r00(x, 20) < 1e-5


def test_full_grid_two_inputs_signed_lags(cyc):
    T, A = 9001, 256
    x = synth.white(T, seed=171).astype(np.complex64)
    y = (np.roll(x, 2) * np.exp(2j * np.pi * 0.25 * np.arange(T))).astype(np.complex64)
    lags = np.arange(-8, 9)
    R, neff = run_full(cyc, x, y, lags, A, [3000, 6001])
    Ro, no = oracle.estimate_xy(x, y, lags, grid(A))
    assert neff == no
    assert np.max(np.abs(R - Ro)) / oracle.r00_xy(x, y, 8, 8) < 1e-5


def test_full_grid_many_lags_wide_span(cyc):
    """Several 16-lag groups per block row, unsorted lags spanning 2560 samples."""
    T, A = 12000, 512
    x = synth.white(T, seed=174).astype(np.complex64)
    lags = np.concatenate([np.arange(0, 40), [2560, 1000, 7, 2047]])
    R, neff = run_full(cyc, x, None, lags, A, [5000, 7000])
    Ro, no = oracle.estimate(x, lags, grid(A))
    assert neff == no
    assert np.max(np.abs(R - Ro)) / oracle.r00(x, 2560) < 1e-5


def test_full_grid_largest_A(cyc):
    T, A = 30011, 4096
    x = synth.white(T, seed=172).astype(np.complex64)
    lags = np.array([0, 5, 31])
    R, neff = run_full(cyc, x, None, lags, A, [T])
    Ro, no = oracle.estimate(x, lags, grid(A))
    assert np.max(np.abs(R - Ro)) / oracle.r00(x, 31) < 1e-5


def test_full_grid_save_load_reset_and_errors(cyc):
    import torch
    T, A = 5000, 128
    x = synth.white(T, seed=173).astype(np.complex64)
    lags = np.array([0, 1, 9])
    Ro, _ = oracle.estimate(x, lags, grid(A))
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    with cyc.Stream(lags, None, 3, full=A) as s1, cyc.Stream(lags, None, 3, full=A) as s2:
        s1.push(xt[:2 * 2222])
        s2.load(s1.save())
        s2.push(xt[2 * 2222:])
        R, _ = s2.read()
        assert np.max(np.abs(R - Ro)) / oracle.r00(x, 9) < 1e-5
        s2.reset()
        s2.push(xt)
        R2, _ = s2.read()
        assert np.max(np.abs(R2 - Ro)) / oracle.r00(x, 9) < 1e-5
    for bad in (100, 8192, 1):
        with pytest.raises(cyc.CycError) as e:
            cyc.Stream(lags, None, 3, full=bad)
        assert e.value.code == cyc.CYC_EINVAL


def test_full_grid_device_host_and_offset_chunks_agree(cyc):
    """Device chunks, host chunks and device chunks whose samples sit at a 4-byte offset
    (not 8-byte aligned) give the same sums through ragged pushes of two inputs, and match
    the oracle."""
    import torch
    T, A = 7001, 128
    x = synth.white(T, seed=175).astype(np.complex64)
    y = synth.white(T, seed=176).astype(np.complex64)
    lags = np.arange(-5, 12)
    chunks = [2, 700, 5, 4000, 2294]
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda()
    xo = torch.zeros(2 * T + 2, device="cuda")         # the same samples at a 4-byte offset
    yo = torch.zeros(2 * T + 2, device="cuda")
    xo[1:2 * T + 1] = xt
    yo[1:2 * T + 1] = yt
    res = []
    for mode in ("device", "host", "offset"):
        with cyc.Stream(lags, None, 3, cross=True, full=A) as s:
            pos = 0
            for c in chunks:
                if mode == "device":
                    s.push(xt[2 * pos:2 * (pos + c)], y=yt[2 * pos:2 * (pos + c)])
                elif mode == "host":
                    s.push(x[pos:pos + c], y=y[pos:pos + c])
                else:
                    s.push(xo.data_ptr() + 4 + 8 * pos, c, 1, y=yo.data_ptr() + 4 + 8 * pos)
                pos += c
            res.append(s.read())
    (R0, n0), (R1, n1), (R2, n2) = res
    assert n0 == n1 == n2
    assert np.array_equal(R0, R1) and np.array_equal(R0, R2)
    Ro, no = oracle.estimate_xy(x, y, lags, grid(A))
    assert n0 == no
    assert np.max(np.abs(R0 - Ro)) / oracle.r00_xy(x, y, 5, 11) < 1e-5


def test_full_grid_many_pushes_fold_in_batches(cyc):
    """Device pushes are folded several at a time (up to 16 chunks or max_chunk samples per
    launch): 40 ragged device pushes with a read in between, a stream whose max_chunk forces
    folds by size, and one interleaving host and device chunks -- all equal to the oracle;
    the interleaved run folds the same batches as the first and equals it bit for bit."""
    import torch
    T, A = 30011, 256
    x = synth.white(T, seed=177).astype(np.complex64)
    lags = np.arange(0, 33)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    rng = np.random.default_rng(178)
    cuts = np.sort(rng.choice(np.arange(1, T), 39, replace=False))
    chunks = np.diff(np.concatenate([[0], cuts, [T]]))
    Ro, no = oracle.estimate(x, lags, grid(A))
    r00 = oracle.r00(x, 32)
    res = []
    for max_chunk in (0, 4096):
        with cyc.Stream(lags, None, 3, full=A, max_chunk=max_chunk) as s:
            pos = 0
            for k, c in enumerate(chunks):
                s.push(xt[2 * pos:2 * (pos + c)])
                pos += c
                if k == 20:                          # a read in the middle folds what is pending
                    Rm, nm = s.read()
                    Rp, npre = oracle.estimate(x[:pos], lags, grid(A))
                    assert nm == npre and np.max(np.abs(Rm - Rp)) / r00 < 1e-5
            R, n = s.read()
        assert n == no and np.max(np.abs(R - Ro)) / r00 < 1e-5, max_chunk
        res.append(R)
    with cyc.Stream(lags, None, 3, full=A) as s:
        pos = 0
        for k, c in enumerate(chunks):
            if k % 3 == 1:
                s.push(x[pos:pos + c])               # host memory
            else:
                s.push(xt[2 * pos:2 * (pos + c)])
            pos += c
            if k == 20:
                s.read()
        R, n = s.read()
    assert n == no and np.max(np.abs(R - Ro)) / r00 < 1e-5
    assert np.array_equal(res[0], R)


@pytest.mark.parametrize("A,hop,cross", [(64, 64, False), (256, 100, True), (32, 1, False), (1024, 512, False)])
def test_full_windows_against_the_oracle(cyc, A, hop, cross):
    """Full mode per window (cyc_create_full_window): window k's A-point spectrum per lag and
    form, window-local phase, element by element against the oracle's windowed estimate on
    the grid -1/2 + kk/A (FP32 tolerance 1e-5 of R^0(0)); the ring read in pieces between
    ragged pushes of device and host chunks; the start index does not move a window's phase;
    the running estimate is kept beside the windows."""
    import torch
    T = {64: 5000, 256: 6001, 32: 700, 1024: 6000}[A]
    x = synth.white(T, seed=180).astype(np.complex64)
    y = synth.white(T, seed=181).astype(np.complex64) if cross else None
    lags = np.arange(-4, 7) if cross else np.arange(0, 9)
    Ro = oracle.windows(x, y, lags, grid(A), A, hop)
    r00 = oracle.r00_xy(x, y, int(max(0, -lags.min())), int(lags.max()))
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda() if cross else None
    rng = np.random.default_rng(182)
    cuts = np.sort(rng.choice(np.arange(1, T), 11, replace=False))
    chunks = np.diff(np.concatenate([[0], cuts, [T]]))
    for n0 in (0, (1 << 33) + 5):
        got = []
        cap = Ro.shape[0] + 1
        with cyc.Stream(lags, None, 3, n0=n0, cross=cross, full=A, window=(A, hop, cap)) as s:
            pos = 0
            for k, c in enumerate(chunks):
                sl = slice(2 * pos, 2 * (pos + c))
                if k % 4 == 3:
                    s.push(x[pos:pos + c], y=y[pos:pos + c] if cross else None)     # host chunk
                else:
                    s.push(xt[sl], y=yt[sl] if cross else None)
                pos += c
                if k % 3 == 0:
                    W, k0 = s.read_windows(cap)
                    assert k0 == sum(len(g) for g in got)
                    got.append(W.copy())
            W, k0 = s.read_windows(cap)
            got.append(W.copy())
            R, n = s.read()
        W = np.concatenate(got)
        assert W.shape == Ro.shape, (W.shape, Ro.shape)
        err = float(np.max(np.abs(W - Ro)) / r00)
        assert err < 1e-5, (n0, err)
        Rs, ns = (oracle.estimate_xy(x, y, lags, grid(A), n0=n0) if cross else
                  oracle.estimate(x, lags, grid(A), n0=n0))
        assert n == ns and np.max(np.abs(R - Rs)) / r00 < 1e-5


def test_full_windows_ring_limit_and_arguments(cyc):
    """A push that would complete more windows than the ring holds fails with CYC_EAGAIN and
    changes nothing; reading frees the room; bad arguments fail with CYC_EINVAL."""
    import torch
    A, hop, cap = 64, 32, 4
    T = 64 + 32 * 10 + 8
    x = synth.white(T, seed=183).astype(np.complex64)
    lags = np.array([0, 1, 8])
    Ro = oracle.windows(x, None, lags, grid(A), A, hop)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    with cyc.Stream(lags, None, 3, full=A, window=(A, hop, cap)) as s:
        s.push(xt[:2 * 180])                                  # windows 0 .. 3 complete: 180 - 8 >= 64 + 32 k
        with pytest.raises(cyc.CycError) as e:
            s.push(xt[2 * 180:])                              # would complete 7 more, 11 unread
        assert e.value.code == cyc.CYC_EAGAIN
        W1, _ = s.read_windows(cap)
        s.push(xt[2 * 180:2 * 240])                           # windows 4, 5
        W2, _ = s.read_windows(cap)
        s.push(xt[2 * 240:2 * 300])                           # windows 6, 7
        W3, _ = s.read_windows(cap)
        s.push(xt[2 * 300:])                                  # windows 8 .. 10
        W4, _ = s.read_windows(cap)
    assert [len(w) for w in (W1, W2, W3, W4)] == [4, 2, 2, 3]
    W = np.concatenate([W1, W2, W3, W4])
    assert W.shape == Ro.shape
    assert np.max(np.abs(W - Ro)) / oracle.r00(x, 8) < 1e-5
    for bad in ((100, 10, 4), (64, 0, 4), (64, 10, 0), (8192, 10, 4)):
        with pytest.raises(cyc.CycError) as e:
            cyc.Stream(lags, None, 3, full=bad[0], window=bad)
        assert e.value.code == cyc.CYC_EINVAL
