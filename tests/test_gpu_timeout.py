"""The bounded waits of the tensor-core projection (GPU): a producer arrival that never
comes -- left out on purpose by the test hook CYC_TEST_WITHHOLD_ARRIVAL -- makes a wait run
out after the stream's budget; the kernel ends (every other wait gives up at once, copies
and tensor-core work in flight are waited for), cyc_sync reports CYC_ETIMEDOUT, and the GPU
stays usable: the next stream matches the oracle.  No fault, trap or hang is involved."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_lost_arrival_times_out_and_the_gpu_stays_usable(cyc, precision, monkeypatch):
    import torch
    x = synth.white(20011, seed=170).astype(np.complex64)
    lags = np.arange(16)
    alphas = -0.5 + np.arange(64) / 64.0
    xd = torch.from_numpy(x.view(np.float32).copy()).cuda()
    monkeypatch.setenv("CYC_TEST_WITHHOLD_ARRIVAL", "1")
    s = cyc.Stream(lags, alphas, cyc.CYC_BOTH, precision=precision)
    monkeypatch.delenv("CYC_TEST_WITHHOLD_ARRIVAL")
    try:
        s.set_wait_budget(100000)              # about 50 microseconds per wait
        t0 = time.perf_counter()
        s.push(xd)
        with pytest.raises(cyc.CycError) as e:
            s.sync()
        assert e.value.code == cyc.CYC_ETIMEDOUT
        assert time.perf_counter() - t0 < 5.0
        with pytest.raises(cyc.CycError):
            cyc.cyc_set_wait_budget(s.h, -1)
    finally:
        s.close()
    # the context is intact: a fresh stream on the same GPU gives the oracle's estimate
    with cyc.Stream(lags, alphas, cyc.CYC_BOTH, precision=precision) as t:
        t.push(xd)
        R, n = t.read()
    Ro, no = oracle.estimate(x, lags, alphas)
    assert n == no
    tol = {"bf16x3": 1e-4, "fp16": 1e-2}[precision]
    assert np.max(np.abs(R - Ro)) / oracle.r00(x, 15) < tol
