"""cyc_estimate_static, the entry point that allocates nothing, against the streaming API.

Some callers cannot allocate device memory when they need an estimate (a real-time
callback that must not call cudaMalloc, a plug-in whose host application owns the device
memory pool); cyc_estimate_static serves them from a fixed device array inside the
library.  Its result must equal what cyc_create / cyc_push / cyc_read give on the same
samples, and the FP64 oracle's, within the FP32 path's tolerance (1e-5 relative to
R^0(0)), on two calls in a row that use different sizes, so that nothing left in the
shared array leaks from the first call into the second; and at the array's limit of 2^20
partial sums, where one FP32 partial per entry takes a whole pass of 2^20 samples.  This
file sorts last so that a stop at its first failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def streaming(cyc, x, lags, alphas, forms, n0):
    with cyc.Stream(lags, alphas, forms, precision="fp32", n0=n0) as s:
        s.push(np.ascontiguousarray(x))
        R, neff = s.read()
    return R, neff


def static(cyc, x, lags, alphas, forms, n0):
    import torch
    F = (1 if forms & 1 else 0) + (1 if forms & 2 else 0)
    xd = torch.from_numpy(x.view(np.float32).copy()).cuda()
    out = torch.full((F, len(alphas), len(lags), 2), float("nan"), dtype=torch.float64, device="cuda")
    neff = cyc.cyc_estimate_static(xd, x.size, lags, alphas, forms, n0, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    return o[..., 0] + 1j * o[..., 1], neff


def test_static_matches_streaming_on_two_calls(cyc):
    cases = [
        # (samples, lags, cycle frequencies, forms, n0): the second is smaller in every
        # dimension and spans two passes of 2^20 samples
        (60013, np.arange(0, 97, 3), -0.5 + np.arange(301) / 301.0, 3, 12345),
        ((1 << 20) + 4099, np.array([5, 0, 2]), np.array([0.125, -0.3, 0.4999, 0.125]), 2, (1 << 40) + 7),
    ]
    for i, (T, lags, alphas, forms, n0) in enumerate(cases):
        x = synth.white(T, seed=200 + i).astype(np.complex64)
        Rs, ns = static(cyc, x, lags, alphas, forms, n0)
        Rr, nr = streaming(cyc, x, lags, alphas, forms, n0)
        assert ns == nr == T - lags.max()
        assert np.all(np.isfinite(Rs))
        r00 = oracle.r00(x, int(lags.max()))
        err = float(np.max(np.abs(Rs - Rr)) / r00)
        assert err < 1e-5, (i, err)
        Ro, no = oracle.estimate(x, lags, alphas, forms, n0=n0)
        assert no == ns
        err_o = float(np.max(np.abs(Rs - Ro)) / r00)
        assert err_o < 1e-5, (i, err_o)


def test_static_at_the_partial_limit_against_the_oracle(cyc):
    """4096 cycle frequencies x 128 lags x 2 forms = 2^20 partial sums: one FP32 partial per
    entry over each pass of 2^20 samples.  Sampled entries against the FP64 oracle,
    including the all-positive mean-power entry a = 0, m = 0."""
    T = (1 << 20) + 300
    x = (synth.white(T, seed=230) * 1.3 + 0.4).astype(np.complex64)
    lags = np.arange(128)
    alphas = -0.5 + np.arange(4096) / 4096.0
    Rs, ns = static(cyc, x, lags, alphas, 3, 0)
    assert ns == T - 127
    r00 = oracle.r00(x, 127)
    rng = np.random.default_rng(231)
    picks = [(0, 2048, 0), (1, 2048, 0), (0, 0, 127)] + [(int(rng.integers(2)), int(rng.integers(4096)),
                                                           int(rng.integers(128))) for _ in range(13)]
    for f, ai, m in picks:
        ref = oracle.entries(x, 127, [f + 1], [alphas[ai]], [m])[0][0]
        err = abs(Rs[f, ai, m] - ref) / r00
        assert err < 1e-5, (f, ai, m, err)


def test_static_rejects_misaligned_buffers(cyc):
    import torch
    x = torch.zeros(2 * 1001, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(cyc.CycError) as e:           # x one float in: 4-byte aligned
        cyc.cyc_estimate_static(x.data_ptr() + 4, 1000, [0, 1], [0.1], 1, 0, out)
    assert e.value.code == cyc.CYC_EINVAL
    with pytest.raises(cyc.CycError) as e:           # out one double in: 8-byte aligned
        cyc.cyc_estimate_static(x, 1000, [0, 1], [0.1], 1, 0, out.data_ptr() + 8)
    assert e.value.code == cyc.CYC_EINVAL


def test_static_rejects_sizes_beyond_its_array(cyc):
    import torch
    x = torch.zeros(2 * 1000, dtype=torch.float32, device="cuda")
    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(cyc.CycError) as e:
        cyc.cyc_estimate_static(x, 1000, [0, 1], np.zeros(4097), 1, 0, out)
    assert e.value.code == cyc.CYC_EINVAL and "4096" in str(e.value)
    with pytest.raises(cyc.CycError) as e:
        cyc.cyc_estimate_static(x, 1000, np.arange(1025), [0.1], 3, 0, out)
    assert e.value.code == cyc.CYC_EINVAL
    with pytest.raises(cyc.CycError) as e:
        cyc.cyc_estimate_static(x, 1000, np.arange(512), np.zeros(2049), 3, 0, out)
    assert e.value.code == cyc.CYC_EINVAL and "partial" in str(e.value)
    with pytest.raises(cyc.CycError) as e:
        cyc.cyc_estimate_static(x, 10, [0, 20], [0.1], 1, 0, out)
    assert e.value.code == cyc.CYC_ENODATA
