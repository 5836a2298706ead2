"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU only).

Error metric: max over (form, a, m) of |R_gpu - R_oracle| / R^0(0), with R^0(0) the
oracle's mean power over the committed samples.  Tolerances: FP32 1e-5, BF16x3 1e-4,
FP16 1e-2 (relative to R^0(0)).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from synth import workloads

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "bf16x3": 1e-4, "fp16": 1e-2}
CONV, CONJ, BOTH = 1, 2, 3


def rel_err(R, Ro, x, M):
    return float(np.max(np.abs(R - Ro)) / oracle.r00(x, M))


def run_gpu(cyc, x, lags, alphas, forms=BOTH, precision="fp32", chunks=None, n0=0, device_input=True,
            max_chunk=0):
    import torch
    with cyc.Stream(lags, alphas, forms, precision=precision, n0=n0, max_chunk=max_chunk) as s:
        xt = torch.from_numpy(x.view(np.float32).copy()).cuda() if device_input else None
        pos = 0
        for c in (chunks or [x.size]):
            if device_input:
                s.push(xt[2 * pos:2 * (pos + c)])
            else:
                s.push(np.ascontiguousarray(x[pos:pos + c]))
            pos += c
        assert pos == x.size
        R, neff = s.read()
    return R, neff


PRECS = ["fp32", "bf16x3", "fp16"]


@pytest.fixture(scope="module")
def cfg1():
    return workloads.config1()


@pytest.mark.parametrize("precision", PRECS)
def test_ragged_small_parity(cyc, precision):
    x = synth.white(5003, seed=101).astype(np.complex64)
    lags = np.array([0, 1, 2, 3, 5, 8, 13, 21, 34])
    alphas = np.random.default_rng(1).uniform(-0.5, 0.5, 37)
    R, neff = run_gpu(cyc, x, lags, alphas, precision=precision)
    Ro, no = oracle.estimate(x, lags, alphas)
    assert neff == no == 5003 - 34
    assert rel_err(R, Ro, x, 34) < TOL[precision]


@pytest.mark.parametrize("precision", PRECS)
def test_several_tiles_each_way(cyc, precision):
    # 300 cycle frequencies (3 tiles of 128, ragged) x 2 forms x 70 lags (140 columns)
    x = synth.white(20011, seed=102).astype(np.complex64)
    lags = np.arange(70)
    alphas = -0.5 + np.arange(300) / 300.0
    R, neff = run_gpu(cyc, x, lags, alphas, precision=precision)
    Ro, _ = oracle.estimate(x, lags, alphas)
    assert rel_err(R, Ro, x, 69) < TOL[precision]


@pytest.mark.parametrize("precision", PRECS)
def test_single_form_and_order(cyc, precision):
    x = synth.white(3000, seed=103).astype(np.complex64)
    lags = np.array([7, 0, 3, 7, 1])            # unsorted, a duplicate, odd column count
    alphas = np.array([0.25, -0.1, 0.3333])
    for forms in (CONV, CONJ):
        R, _ = run_gpu(cyc, x, lags, alphas, forms=forms, precision=precision)
        Ro, _ = oracle.estimate(x, lags, alphas, forms)
        assert R.shape == (1, 3, 5)
        assert rel_err(R, Ro, x, 7) < TOL[precision]
        assert np.array_equal(R[0, :, 0], R[0, :, 3])


@pytest.mark.parametrize("precision", PRECS)
def test_chunk_split_invariance(cyc, precision):
    x = synth.white(9000, seed=104).astype(np.complex64)
    lags = np.arange(0, 40, 3)              # M = 39
    alphas = np.linspace(-0.5, 0.5, 23, endpoint=False)
    R1, n1 = run_gpu(cyc, x, lags, alphas, precision=precision)
    splits = [1, 38, 39, 40, 2, 7, 997, 13, 4096, 1, 1]
    splits.append(x.size - sum(splits))
    R2, n2 = run_gpu(cyc, x, lags, alphas, chunks=splits, precision=precision)
    Ro, no = oracle.estimate(x, lags, alphas)
    assert n1 == n2 == no
    tol = TOL[precision]
    assert rel_err(R2, Ro, x, 39) < tol
    assert rel_err(R2, R1, x, 39) < tol / 5
    # pushes longer than max_chunk are cut inside the library
    R3, _ = run_gpu(cyc, x, lags, alphas, max_chunk=1000, precision=precision)
    assert rel_err(R3, Ro, x, 39) < tol


@pytest.mark.parametrize("precision", PRECS)
def test_staged_passes(cyc, precision):
    """Pushes are staged behind each other and projected once max_chunk samples are staged
    or the stream is read: ragged device and host pushes that fill passes of 1000 samples
    several at a time and cross their boundaries, with reads (each runs what is staged)
    between them, give the oracle's estimate of everything pushed so far at every read."""
    import torch
    x = synth.white(9000, seed=112).astype(np.complex64)
    lags = np.arange(0, 40, 3)
    alphas = np.linspace(-0.5, 0.5, 23, endpoint=False)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    splits = [1, 38, 39, 40, 2, 7, 997, 13, 1500, 1, 1, 333, 2999]
    splits.append(x.size - sum(splits))
    tol = TOL[precision]
    with cyc.Stream(lags, alphas, BOTH, precision=precision, max_chunk=1000) as s:
        pos = 0
        for k, c in enumerate(splits):
            if k % 3 == 2:
                s.push(np.ascontiguousarray(x[pos:pos + c]))
            else:
                s.push(xt[2 * pos:2 * (pos + c)])
            pos += c
            if k in (3, 6, 9) and pos > 39:
                R, n = s.read()
                Ro, no = oracle.estimate(x[:pos], lags, alphas)
                assert n == no and rel_err(R, Ro, x[:pos], 39) < tol, k
        R, n = s.read()
    Ro, no = oracle.estimate(x, lags, alphas)
    assert n == no and rel_err(R, Ro, x, 39) < tol


@pytest.mark.parametrize("precision", PRECS)
def test_large_start_index(cyc, precision):
    x = synth.white(4000, seed=105).astype(np.complex64)
    lags = np.arange(6)
    alphas = np.array([0.1, -0.33, 0.123456789, 0.5, 1 / 3.0, 0.0])
    n0 = (1 << 40) + 12345
    R, _ = run_gpu(cyc, x, lags, alphas, n0=n0, precision=precision)
    Ro, _ = oracle.estimate(x, lags, alphas, n0=n0)
    assert rel_err(R, Ro, x, 5) < TOL[precision]


def test_aliases_are_deduplicated(cyc):
    x = synth.white(2500, seed=106).astype(np.complex64)
    alphas = np.array([0.125, 1.125, -0.875, 0.25, 0.125])
    R, _ = run_gpu(cyc, x, [0, 2], alphas)
    assert np.array_equal(R[:, 0], R[:, 1]) and np.array_equal(R[:, 0], R[:, 2]) and np.array_equal(R[:, 0], R[:, 4])
    h = cyc.cyc_create_ex([0, 2], alphas)
    try:
        assert cyc.cyc_info(h)[1] == 2
    finally:
        cyc.cyc_destroy(h)


def test_host_device_inputs_and_outputs(cyc):
    import torch
    x = synth.white(6000, seed=107).astype(np.complex64)
    lags, alphas = np.arange(9), np.array([0.0, 0.2, -0.45])
    Rd, _ = run_gpu(cyc, x, lags, alphas, device_input=True, chunks=[1000, 5000])
    Rh, _ = run_gpu(cyc, x, lags, alphas, device_input=False, chunks=[1000, 5000])
    assert np.array_equal(Rd, Rh)
    with cyc.Stream(lags, alphas) as s:
        s.push(np.ascontiguousarray(x[:1000]))
        s.push(np.ascontiguousarray(x[1000:]))
        out = torch.zeros((2, 3, 9, 2), dtype=torch.float64, device="cuda")
        _, neff = s.read(out)
        torch.cuda.synchronize()
        Rdev = out.cpu().numpy()
    assert neff == 6000 - 8
    assert np.array_equal(Rdev[..., 0] + 1j * Rdev[..., 1], Rh)


def test_save_load_resume(cyc):
    x = synth.white(7000, seed=108).astype(np.complex64)
    lags, alphas = np.arange(0, 30, 2), np.linspace(-0.5, 0.5, 11)
    with cyc.Stream(lags, alphas) as s0:         # the same passes: a sync runs what is staged
        s0.push(np.ascontiguousarray(x[:2500]))
        s0.sync()
        s0.push(np.ascontiguousarray(x[2500:]))
        Rfull, _ = s0.read()
    with cyc.Stream(lags, alphas) as s:
        s.push(np.ascontiguousarray(x[:2500]))
        blob = s.save()
    with cyc.Stream(lags, alphas) as s2:
        s2.load(blob)
        s2.push(np.ascontiguousarray(x[2500:]))
        R2, _ = s2.read()
    assert np.array_equal(R2, Rfull)
    with cyc.Stream(lags, alphas[:5]) as s3:
        with pytest.raises(cyc.CycError) as e:
            s3.load(blob)
        assert e.value.code == -1


def test_reset_and_nodata_and_errors(cyc):
    x = synth.white(100, seed=109).astype(np.complex64)
    with cyc.Stream([0, 50], [0.1]) as s:
        s.push(np.ascontiguousarray(x[:40]))
        out = np.full((2, 1, 2), 7.0 + 7.0j)
        with pytest.raises(cyc.CycError) as e:
            s.read(out)
        assert e.value.code == -6 and np.all(out == 7.0 + 7.0j)
        s.push(np.ascontiguousarray(x[40:]))
        R1, n = s.read()
        assert n == 50
        s.reset()
        assert s.info()[2:] == (0, 0)
        s.push(np.ascontiguousarray(x))
        R2, _ = s.read()
        assert np.array_equal(R1, R2)
        with pytest.raises(cyc.CycError):
            s.push(np.ascontiguousarray(x), nsamples=-1)
    for bad in (dict(lags=[-(1 << 21), 2], alphas=[0.1]), dict(lags=[], alphas=[0.1]), dict(lags=[1], alphas=[]),
                dict(lags=[1], alphas=[float("nan")]), dict(lags=[1], alphas=[0.1], conj_flag=4)):
        with pytest.raises(cyc.CycError) as e:
            cyc.cyc_create_ex(**bad)
        assert e.value.code == -1


def test_config0_full_grid(cyc):
    w = workloads.config0()
    x, lags = w["x"], w["lags"]
    for forms, al in ((CONV, w["alphas_conv"]), (CONJ, w["alphas_conj"])):
        R, neff = run_gpu(cyc, x, lags, al, forms=forms)
        Ro, no = oracle.estimate(x, lags, al, forms)
        assert neff == no == 65536 - 31
        assert rel_err(R, Ro, x, 31) < 1e-5


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_config1_full_size_sampled(cyc, cfg1, precision):
    """2^26 samples in 2^16 chunks, 1024 cycle frequencies, 128 lags, both forms; the
    oracle recomputes 12 sampled entries over all 2^26 - 127 terms."""
    w = cfg1
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    C = w["chunk"]
    R, neff = run_gpu(cyc, x, lags, alphas, chunks=[C] * (x.size // C), precision=precision)
    assert neff == x.size - 127
    rng = np.random.default_rng(7)
    f = rng.integers(0, 2, 12)
    ia = rng.integers(0, 1024, 12)
    im = rng.integers(0, 128, 12)
    f[0], ia[0], im[0] = 0, 512, 0                  # a = 0, m = 0: the mean power itself
    f[1], ia[1], im[1] = 0, 1023, 127               # last row, last column
    Ro, _ = oracle.entries(x, 127, f + 1, alphas[ia], lags[im])
    r00 = oracle.r00(x, 127)
    err = np.max(np.abs(R[f, ia, im] - Ro)) / r00
    assert err < TOL[precision]
    assert abs(R[0, 512, 0] - r00) / r00 < TOL[precision]


@pytest.mark.parametrize("precision", PRECS)
def test_config2_full_size_sampled(cyc, precision):
    """One 2^20-sample block, 4096 cycle frequencies, 256 lags, both forms (two column
    tiles for the tensor-core path); 24 sampled entries plus the strongest conjugate line."""
    w = workloads.config2()
    x, lags, alphas = w["x"], w["lags"], w["alphas"]
    R, neff = run_gpu(cyc, x, lags, alphas, precision=precision)
    assert neff == x.size - 255
    rng = np.random.default_rng(11)
    f = rng.integers(0, 2, 24)
    ia = rng.integers(0, 4096, 24)
    im = rng.integers(0, 256, 24)
    # conjugate line of GMSK at 4 sps: 2 f0 + 1/8 -> nearest grid index
    k = int(round(((2 * w["f0"] + 0.125 + 0.5) % 1.0) * 4096)) % 4096
    f[0], ia[0], im[0] = 1, k, 0
    f[1], ia[1], im[1] = 1, 4095, 255
    f[2], ia[2], im[2] = 0, 2048, 0                 # a = 0, m = 0: the mean power itself
    Ro, _ = oracle.entries(x, 255, f + 1, alphas[ia], lags[im])
    err = np.max(np.abs(R[f, ia, im] - Ro)) / oracle.r00(x, 255)
    assert err < TOL[precision], err


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_tensor_core_lag_limit(cyc, precision):
    """Lags up to 2560 stage through shared memory in blocks with their halo; beyond that
    the tensor-core projection declines (CYC_ENOTSUP) and FP32 serves."""
    x = synth.white(30011, seed=110).astype(np.complex64)
    lags = np.array([0, 1, 999, 2560, 7])
    alphas = np.array([0.0, 0.21, -0.4, 0.33])
    R, neff = run_gpu(cyc, x, lags, alphas, precision=precision, chunks=[5000, 9000, 16011])
    Ro, no = oracle.estimate(x, lags, alphas)
    assert neff == no
    assert rel_err(R, Ro, x, 2560) < TOL[precision]
    with pytest.raises(cyc.CycError) as e:
        cyc.Stream([0, 2561], [0.1], cyc.CYC_BOTH, precision=precision)
    assert e.value.code == cyc.CYC_ENOTSUP


@pytest.mark.parametrize("na", [1, 2, 5, 8, 16, 17, 32, 33])
def test_fp32_small_and_general_paths(cyc, na):
    """FP32 with at most 32 distinct cycle frequencies takes the register/warp-shuffle path
    (classes of 1, 2, 4, 8, 16, 32), 33 and more the GEMM-tiled one; both match the oracle on
    ragged column counts."""
    x = synth.white(12007, seed=111).astype(np.complex64)
    lags = np.array([0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89])
    alphas = np.linspace(-0.45, 0.45, na) if na > 1 else np.array([0.2])
    R, neff = run_gpu(cyc, x, lags, alphas, chunks=[3001, 9006])
    Ro, no = oracle.estimate(x, lags, alphas)
    assert neff == no
    assert rel_err(R, Ro, x, 89) < 1e-5


@pytest.mark.parametrize("na", [1, 2, 3, 6, 12, 20, 31])
def test_register_sum_passes(cyc, na):
    """The register-sum path updates the FP64 sums and copies the carried tail inside its one
    launch (the last block of each column group adds the splits; its arrival counter is reset
    for the next launch): many short passes (max_chunk 700, ragged pushes, reads in between),
    one input and two, every block shape, each read against the oracle."""
    import torch
    T = 6000
    x = synth.white(T, seed=113 + na).astype(np.complex64)
    y = (0.6 * np.roll(x, 5) + 0.8 * synth.white(T, seed=213 + na)).astype(np.complex64)
    lags = np.array([-7, 0, 1, 4, 9, 30])
    alphas = np.random.default_rng(114 + na).uniform(-0.5, 0.5, na)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    yt = torch.from_numpy(y.view(np.float32).copy()).cuda()
    cuts = [0, 1, 699, 700, 1901, 2500, 4444, T]
    for cross in (False, True):
        with cyc.Stream(lags, alphas, BOTH, precision="fp32", max_chunk=700, cross=cross) as s:
            for k in range(len(cuts) - 1):
                a, b = cuts[k], cuts[k + 1]
                s.push(xt[2 * a:2 * b], y=yt[2 * a:2 * b] if cross else None)
                if b in (1901, 4444, T):
                    R, n = s.read()
                    Ro, no = oracle.estimate_xy(x[:b], y[:b] if cross else None, lags, alphas)
                    nrm = oracle.r00_xy(x[:b], y[:b] if cross else None, 7, 30)
                    assert n == no and np.max(np.abs(R - Ro)) / nrm < 1e-5, (cross, b)


def test_reset_on_the_register_sum_path(cyc):
    """A reset of a register-sum stream leaves the zeroing of the sums to its next pass (which
    writes its totals instead of adding them) or to whatever reads the sums first: after
    resets, reads, raw sums, save/load and pushes too short to commit a term see exactly the
    samples pushed since the last reset."""
    import torch
    T = 5000
    x = synth.white(T, seed=118).astype(np.complex64)
    lags = np.array([0, 2, 5, 11])
    alphas = np.array([0.0, 0.125, -0.3, 0.41, 0.07])
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()

    def want(lo, hi):
        Ro, no = oracle.estimate(x[lo:hi], lags, alphas, n0=0)
        return Ro, no, oracle.r00(x[lo:hi], 11)

    with cyc.Stream(lags, alphas, BOTH, precision="fp32", max_chunk=1500) as s:
        s.push(xt[:2 * 2000])
        R, n = s.read()
        Ro, no, r0 = want(0, 2000)
        assert n == no and np.max(np.abs(R - Ro)) / r0 < 1e-5
        s.reset()                                   # the next pass writes its totals
        s.push(xt[2 * 2000:2 * 4500])               # two passes (max_chunk 1500)
        R, n = s.read()
        Ro, no, r0 = want(2000, 4500)
        assert n == no and np.max(np.abs(R - Ro)) / r0 < 1e-5
        s.reset()                                   # read before any pass: zeroed by the read
        raw, n = s.sums()
        assert n == 0 and float(raw.abs().max()) == 0.0
        s.push(xt[2 * 4500:2 * 4505])               # 5 samples: fewer than max(lags) + 1
        with pytest.raises(cyc.CycError) as e:
            s.read()
        assert e.value.code == cyc.CYC_ENODATA
        s.reset()
        blob = s.save()                             # save right after a reset: zero sums
        s.push(xt[:2 * 3000])
        s.load(blob)
        s.push(xt[2 * 1000:2 * 2500])
        R, n = s.read()
        Ro, no, r0 = want(1000, 2500)
        assert n == no and np.max(np.abs(R - Ro)) / r0 < 1e-5


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_tensor_core_unit_kinds(cyc, precision):
    """The tensor-core projection takes a and -a together (one pair of weight rows), 0 and
    1/2 as one unit of real rows, and every other a alone: symmetric grids, grids without
    a = 0 or 1/2, one-sided random sets, their mix with duplicates and aliases, several
    units tiles (pairs of CTAs, the odd CTA sometimes empty), two column tiles and a ragged
    last column tile, all against the oracle."""
    rng = np.random.default_rng(40)
    cases = [
        (9001, np.arange(128), -0.5 + np.arange(512) / 512),                 # 255 pairs + {0, 1/2}
        (7003, np.arange(41), (np.arange(130) - 64.5) / 130),                # 65 pairs, no self-conjugate a
        (6007, np.arange(200), rng.uniform(0.01, 0.49, 129)),                # 129 singles, 2 column tiles
        (5003, np.arange(64), np.concatenate([[0.0], rng.uniform(-0.5, 0.5, 40), [0.5]])),
        (4001, np.arange(100), np.concatenate([-0.5 + np.arange(300) / 300, [0.25, 1.25, -0.75, 0.1]])),
        (3001, np.array([0, 3, 1, 3, 17]), np.array([0.5, -0.5, 0.0, 1.0, 0.3, -0.3, 0.7])),
    ]
    for i, (T, lags, alphas) in enumerate(cases):
        x = synth.white(T, seed=120 + i).astype(np.complex64)
        Ro, no = oracle.estimate(x, lags, alphas)
        R, neff = run_gpu(cyc, x, lags, alphas, precision=precision, chunks=[T // 3, T - T // 3])
        assert neff == no
        assert rel_err(R, Ro, x, int(lags.max())) < TOL[precision], i


@pytest.mark.parametrize("precision", PRECS)
def test_long_single_push_accumulation(cyc, precision):
    """One push of 2^20 + 100 samples: every FP32 accumulation chain (tensor-memory or
    register sums) is bounded, so even the all-positive mean-power entry a = 0, m = 0 keeps
    its tolerance; 20 cycle frequencies so that FP32 takes the GEMM path."""
    T = (1 << 20) + 100
    x = (synth.white(T, seed=130) * 1.3 + 0.4).astype(np.complex64)
    lags = np.array([0, 1, 7, 100])
    alphas = np.concatenate([[0.0], np.random.default_rng(30).uniform(-0.5, 0.5, 19)])
    R, neff = run_gpu(cyc, x, lags, alphas, precision=precision)
    Ro, no = oracle.estimate(x, lags, alphas)
    assert neff == no
    r00 = oracle.r00(x, 100)
    assert abs(R[0, 0, 0] - r00) / r00 < TOL[precision] / 4
    assert rel_err(R, Ro, x, 100) < TOL[precision]
