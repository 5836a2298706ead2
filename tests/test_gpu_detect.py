"""cyc_detect (cycle-frequency detection on a stream's estimate, Sec. 6's next step) against
the oracle's rule, element by element, through the C ABI (GPU only); and the proposer's
fallback run end to end: a proposal with confidence below tau sends the caller to the full
grid, whose detections are the rule applied to the full-grid estimate."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import detect as od

pytestmark = pytest.mark.gpu

A = 128
GRID = -0.5 + np.arange(A) / A


def gmsk(T, f0=3 / 128, sps=8, snr=20.0, seed=0xC7C1_0D01):
    s = synth.carrier(synth.gmsk(T, bt=0.3, sps=sps, seed=seed), f0)
    return synth.add_awgn(s, snr, seed=seed).astype(np.complex64)


def same_rule(flags, ratio, R, alphas, forms=(1, 2)):
    """The library's flags equal the oracle rule applied to the same estimate R."""
    det, rat, lm = od.cfar(R, alphas, forms)
    assert np.array_equal(flags & 1, det.astype(np.uint8))
    assert np.array_equal((flags >> 1) & 1, lm.astype(np.uint8))
    ok = np.isfinite(rat) & (rat < 1e30)
    assert np.allclose(ratio[ok], rat[ok], rtol=1e-6, atol=0.0)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_detect_matches_rule_on_gmsk(cyc, precision):
    x = gmsk((1 << 17) + 31)
    lags = np.arange(16)
    with cyc.Stream(lags, GRID, cyc.CYC_BOTH, precision=precision) as s:
        s.push(x)
        R, _ = s.read()
        flags, ratio, nd = s.detect()
    same_rule(flags, ratio, R, GRID)
    assert nd == int((flags & 1).sum())
    # the four lines of the signal (conventional +-1/T, conjugate 2 f0 +- 1/(2T)) are found,
    # as on the FP64 oracle's own estimate
    Ro, _ = oracle.estimate(x, lags, GRID)
    det_o, _, _ = od.cfar(Ro, GRID)
    k = lambda a: int(round((a + 0.5) * A)) % A          # noqa: E731
    for f, lines in ((0, [k(1 / 8), k(-1 / 8)]), (1, [k(3 / 64 + 1 / 16), k(3 / 64 - 1 / 16)])):
        assert (flags[f, lines] & 1).all() and det_o[f, lines].all(), f


def test_detect_device_outputs_single_form_and_errors(cyc):
    import torch
    x = gmsk((1 << 15) + 7, seed=0xC7C1_0D02)
    lags = np.arange(0, 24, 3)
    alphas = GRID[::-1].copy()                      # any order: the list is the circular grid
    with cyc.Stream(lags, alphas, cyc.CYC_CONJ) as s:
        with pytest.raises(cyc.CycError) as e:
            s.detect()
        assert e.value.code == cyc.CYC_ENODATA
        s.push(x)
        R, _ = s.read()
        fd = torch.zeros((1, A), dtype=torch.uint8, device="cuda")
        rd = torch.zeros((1, A), dtype=torch.float32, device="cuda")
        s.detect(8.4, 12, fd, rd)
        det, rat, lm = od.cfar(R, alphas, (2,), win=12)
        assert np.array_equal(fd.cpu().numpy() & 1, det.astype(np.uint8))
        assert np.allclose(rd.cpu().numpy(), rat, rtol=1e-6)
        for kappa, win in ((0.0, 16), (8.4, 1), (8.4, 33), (float("nan"), 16)):
            with pytest.raises(cyc.CycError) as e:
                s.detect(kappa, win)
            assert e.value.code == cyc.CYC_EINVAL


def test_detect_full_mode_stream(cyc):
    x = gmsk((1 << 16) + 15, seed=0xC7C1_0D03)
    lags = np.arange(8)
    with cyc.Stream(lags, None, cyc.CYC_BOTH, full=A) as s:
        s.push(x)
        R, _ = s.read()
        flags, ratio, _ = s.detect()
    same_rule(flags, ratio, R, GRID)


def test_proposer_fallback_runs_the_full_grid(cyc):
    """tau = 1 makes every proposal fall back (confidence is below 1); the caller then runs
    the full 512-point grid and takes cyc_detect's detections, which are the oracle rule on
    that estimate and contain the signal's lines."""
    import torch
    from paper_2405_16911_gb300 import proposer_train as pt
    if not os.path.exists(pt.WEIGHTS):
        pytest.skip("no trained weights committed")
    x = gmsk(pt.NS, f0=5 / 512, sps=8, seed=0xC7C1_0D04)
    xd = torch.from_numpy(x.view(np.float32)).cuda()
    net = cyc.cyc_net_create(np.load(pt.WEIGHTS), 0)
    try:
        ac, aj, conf, fb = cyc.cyc_propose(net, xd, pt.NS, k=32, tau=1.0)
        assert fb == 1 and conf < 1.0
        ac2, aj2, conf2, fb2 = cyc.cyc_propose(net, xd, pt.NS, k=32, tau=0.0)
        assert fb2 == 0 and conf2 == conf
    finally:
        cyc.cyc_net_destroy(net)
    with cyc.Stream(pt.LAGS, pt.GRID, cyc.CYC_BOTH, precision="bf16x3", max_chunk=pt.NS) as s:
        s.push(xd)
        R, _ = s.read()
        flags, ratio, nd = s.detect(pt.KAPPA)
    same_rule(flags, ratio, R, pt.GRID)
    k = lambda a: int(round((a + 0.5) * 512)) % 512      # noqa: E731
    assert flags[0, k(1 / 8)] & 1 and flags[0, k(-1 / 8)] & 1
    assert flags[1, k(10 / 512 + 1 / 16)] & 1 and flags[1, k(10 / 512 - 1 / 16)] & 1
    assert nd >= 4
