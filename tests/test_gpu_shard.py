"""Time shards of one stream, each estimated by its own libcyc stream, merged (GPU).

On one GPU the shards run one after another; on several GPUs each rank runs one, and
the merge is the single all-reduce of shard.allreduce_merge.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_2405_16911_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16x3", 1e-4)])
def test_shards_merge_to_the_whole_stream(cyc, precision, tol):
    T, lags = 50021, np.arange(0, 64, 5)
    M = int(lags.max())
    alphas = -0.5 + np.arange(200) / 200.0
    x = synth.white(T, seed=300).astype(np.complex64)
    res = []
    for s0, s1, a, cnt in shard.time_shards(T, M, 3):
        with cyc.Stream(lags, alphas, cyc.CYC_BOTH, precision=precision, n0=a) as s:
            s.push(np.ascontiguousarray(x[s0:s1]))
            R, n = s.read()
            assert n == cnt
        res.append((R, n))
    Rm, nm = shard.merge(res)
    Ro, no = oracle.estimate(x, lags, alphas)
    assert nm == no
    assert np.max(np.abs(Rm - Ro)) / oracle.r00(x, M) < tol


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16x3", 1e-4)])
def test_raw_sums_merge_in_place(cyc, precision, tol):
    """The merge that shard.allreduce_stream does across GPUs, on one GPU: the shards'
    device running sums (cyc_sums) added in place into one handle's, its count set to the
    total (cyc_set_n_eff), and the library's own read gives the whole stream's estimate."""
    import torch
    T, lags = 40013, np.array([0, 2, 9, 31])
    M = 31
    alphas = np.concatenate([-0.5 + np.arange(256) / 256.0, [0.123]])
    x = synth.white(T, seed=301).astype(np.complex64)
    streams = []
    try:
        for s0, s1, a, cnt in shard.time_shards(T, M, 3):
            s = cyc.Stream(lags, alphas, cyc.CYC_BOTH, precision=precision, n0=a)
            s.push(np.ascontiguousarray(x[s0:s1]))
            streams.append(s)
        views = [s.sums() for s in streams]
        total = sum(n for _, n in views)
        for v, _ in views[1:]:
            views[0][0].add_(v)
        torch.cuda.synchronize()
        streams[0].set_n_eff(total)
        R, n = streams[0].read()
    finally:
        for s in streams:
            s.close()
    Ro, no = oracle.estimate(x, lags, alphas)
    assert n == no == total
    assert np.max(np.abs(R - Ro)) / oracle.r00(x, M) < tol
