"""The tensor-core precisions against an FP64 emulation of their operand rounding (GPU).

The GPU's error against the exact FP64 oracle must be of the size the emulated operand
rounding predicts: a kernel that dropped the lo parts (single-pass bf16) would be about 2^8
times worse, one that skipped the rounding (FP32 operands) far better.  Entry by entry the
two cannot agree more closely than the rounding of the lo parts allows: the kernel's FP32
weights differ from exact ones by ~1e-6, which moves some lo parts by one bf16 step."""
import numpy as np
import pytest

import oracle
import synth
from oracle import split

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16x3", "fp16"])
def test_gpu_error_has_the_size_of_its_operand_rounding(cyc, precision):
    import torch
    x = synth.white(48, seed=150).astype(np.complex64)
    lags = np.array([0, 3, 7])
    alphas = np.random.default_rng(50).uniform(-0.5, 0.5, 20)
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    with cyc.Stream(lags, alphas, 3, precision=precision) as s:
        s.push(xt)
        R, neff = s.read()
    Ro, no = oracle.estimate(x, lags, alphas)
    Re, ne = split.estimate_rounded(x, lags, alphas, precision=precision)
    assert neff == no == ne == 41
    e_round = np.max(np.abs(Re - Ro))          # what the operand rounding alone costs
    e_gpu = np.max(np.abs(R - Ro))
    assert e_round > {"bf16x3": 1e-7, "fp16": 1e-5}[precision]
    assert e_round / 3 < e_gpu < 3 * e_round, (e_gpu, e_round)
