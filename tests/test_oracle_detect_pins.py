"""Pins of oracle.detect (the cycle-frequency detection rule, Sec. 6's next step) to things
other than itself: constructed statistics where each clause of the rule decides the outcome
(the noise window leaves out +-1, the even-count median, the circular neighbourhood, the
local maximum, the excluded conventional a = 0), a tone's single conjugate line, GMSK's
line locations (Sec. 3), and white noise without false alarms."""
import numpy as np

import oracle
import synth
from oracle import detect

CONV, CONJ = 1, 2
A = 64
GRID = -0.5 + np.arange(A) / A


def R_from_s(s_conj, s_conv=None):
    """An estimate [2][A][1] whose statistic is s (one lag: |R|^2 = s)."""
    s_conv = np.ones(A) if s_conv is None else s_conv
    return np.stack([np.sqrt(s_conv), np.sqrt(s_conj)]).astype(np.complex128)[:, :, None]


def test_noise_window_leaves_out_the_neighbours():
    s = np.ones(A)                 # perfect squares throughout, so |sqrt(s)|^2 == s exactly
    s[10] = 400.0
    for d in range(2, 10):
        s[10 + d] = s[10 - d] = 64.0
    det, ratio, lm = detect.cfar(R_from_s(s), GRID, kappa=8.4)
    # offsets +-2..+-16: 16 values of 64 and 14 of 1 -> median 64, ratio exactly 6.25 (with
    # +-1 in the window: 16 and 16 -> median 32.5, ratio 12.3, detected)
    assert ratio[1, 10] == 6.25
    assert not det[1, 10]
    det, _, _ = detect.cfar(R_from_s(s), GRID, kappa=6.0)
    assert det[1, 10]


def test_even_count_median_is_the_mean_of_the_middle_pair():
    s = np.ones(A)
    for d in range(2, 17):
        s[40 + d] = 9.0            # 15 values of 9 on one side, 15 of 1 on the other
    s[40] = 25.0
    s[39] = s[41] = 1.0
    _, ratio, _ = detect.cfar(R_from_s(s), GRID)
    assert ratio[1, 40] == 5.0     # median (1 + 9) / 2 = 5


def test_neighbourhood_wraps_around_the_grid():
    s = np.ones(A)
    for d in range(2, 17):
        s[(0 - d) % A] = 49.0
    s[0] = 400.0
    _, ratio, _ = detect.cfar(R_from_s(s), GRID)
    assert ratio[1, 0] == 16.0     # median of 15 x 49 and 15 x 1 = 25


def test_only_local_maxima_are_detected():
    s = np.ones(A)
    s[20], s[21] = 100.0, 121.0
    s[30] = s[31] = 100.0
    det, ratio, lm = detect.cfar(R_from_s(s), GRID)
    assert ratio[1, 20] > 8.4 and not det[1, 20]
    assert det[1, 21] and det[1, 30] and det[1, 31]
    assert det[1].sum() == 3


def test_conventional_dc_line_is_excluded():
    s = np.ones(A)
    s[32] = 1e6                    # a = 0 on this grid
    det, ratio, _ = detect.cfar(R_from_s(s, s_conv=s.copy()), GRID)
    assert det[1, 32] and not det[0, 32] and ratio[0, 32] == 0.0
    assert det[0].sum() == 0


def test_tone_conjugate_line_dominates():
    """A tone at f0 has its conjugate line at 2 f0 (|R| = 1 at every lag) and, with N_eff a
    multiple of the grid period, nothing else on the grid but the noise; its ratio exceeds
    every other bin's of both forms by orders of magnitude."""
    f0 = 3 / A
    T = 64 * 300 + 7
    x = (synth.tone(T, f0) + 1e-3 * synth.white(T, seed=901)).astype(np.complex64)
    lags = np.arange(8)
    R, _ = oracle.estimate(x, lags, GRID)
    det, ratio, _ = detect.cfar(R, GRID)
    line = 32 + 6                                         # a = 2 f0
    assert det[1, line]
    others = np.concatenate([np.delete(ratio[1], line), ratio[0]])
    assert ratio[1, line] > 1e6 * others.max()


def test_gmsk_lines_are_detected_and_dominate():
    """GMSK (h = 1/2) at 20 dB: conventional lines at +-1/T, conjugate lines at 2 f0 +- 1/(2T)
    (Sec. 3), detected with the two largest ratios of their form, five times any other
    detection's (the others sit where the estimator's own noise floor peaks: near a = 0
    for the conventional form and near 2 f0 for the conjugate one)."""
    sps, f0, A2 = 8, 3 / 128, 128
    grid = -0.5 + np.arange(A2) / A2
    T = (1 << 17) + 31
    s = synth.carrier(synth.gmsk(T, bt=0.3, sps=sps, seed=0xC7C1_0D01), f0)
    x = synth.add_awgn(s, 20.0, seed=0xC7C1_0D01).astype(np.complex64)
    R, _ = oracle.estimate(x, np.arange(16), grid)
    det, ratio, _ = detect.cfar(R, grid)
    k = lambda a: int(round((a + 0.5) * A2)) % A2          # noqa: E731
    for f, lines in ((0, [k(1 / sps), k(-1 / sps)]), (1, [k(2 * f0 + 0.5 / sps), k(2 * f0 - 0.5 / sps)])):
        assert det[f, lines].all(), f
        rest = np.delete(np.where(det[f], ratio[f], 0.0), lines)
        assert ratio[f, lines].min() > 5 * rest.max(), f


def test_white_noise_gives_no_detections():
    grid = -0.5 + np.arange(256) / 256
    total = 0
    for seed in range(8):
        x = synth.white((1 << 14) + 31, seed=0xC7C1_0D10 + seed).astype(np.complex64)
        R, _ = oracle.estimate(x, np.arange(32), grid)
        det, ratio, _ = detect.cfar(R, grid)
        total += int(det.sum())
        assert np.isfinite(ratio).all()
    assert total == 0
