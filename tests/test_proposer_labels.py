"""The proposer's label rule (the constant-false-alarm detection of oracle.detect, which
cyc_detect implements in the library) on synthetic estimates of the label grid."""
import numpy as np

from oracle import detect as od

GRID = -0.5 + np.arange(512) / 512.0


def noise(rng, scale=1.0):
    return scale * (rng.normal(size=(2, 512, 64)) + 1j * rng.normal(size=(2, 512, 64)))


def test_few_false_alarms_on_noise_even_when_its_level_varies_with_a():
    rng = np.random.default_rng(0)
    bumps = 1.0 + 30.0 * np.exp(-0.5 * ((np.arange(512) - 256) / 20.0) ** 2)   # noise piled near a = 0
    fa = 0
    for _ in range(100):
        R = noise(rng) * np.sqrt(bumps)[None, :, None]
        fa += od.cfar(R, GRID)[0].sum()
    assert fa / 100 < 0.05


def test_planted_lines_are_detected_and_the_a0_line_is_not():
    rng = np.random.default_rng(1)
    R = noise(rng, 0.01)
    R[0, 256, :] += 5.0                           # conventional a = 0: always present, never a label
    R[0, 320, 10] += 0.2                          # a = 1/8 at lag 10
    R[1, 100, 0] += 0.3
    lab = od.cfar(R, GRID)[0]
    assert lab[0, 320] and lab[1, 100]
    assert not lab[0, 256]
    assert lab.sum() <= 3
