"""The proposer's label rule (local constant-false-alarm detection) on synthetic estimates."""
import numpy as np

from paper_2405_16911_gb300 import proposer_train as pt


def noise(rng, scale=1.0):
    return scale * (rng.normal(size=(2, 512, 64)) + 1j * rng.normal(size=(2, 512, 64)))


def test_few_false_alarms_on_noise_even_when_its_level_varies_with_a():
    rng = np.random.default_rng(0)
    bumps = 1.0 + 30.0 * np.exp(-0.5 * ((np.arange(512) - 256) / 20.0) ** 2)   # noise piled near a = 0
    fa = 0
    for _ in range(100):
        R = noise(rng) * np.sqrt(bumps)[None, :, None]
        fa += pt.detect(R, 65536).sum()
    assert fa / 100 < 0.05


def test_planted_lines_are_detected_and_the_a0_line_is_not():
    rng = np.random.default_rng(1)
    R = noise(rng, 0.01)
    R[0, 256, :] += 5.0                           # conventional a = 0: always present, never a label
    R[0, 320, 10] += 0.2                          # a = 1/8 at lag 10
    R[1, 100, 0] += 0.3
    lab = pt.detect(R, 65536)
    assert lab[0, 320] == 1 and lab[1, 100] == 1
    assert lab[0, 256] == 0
    assert lab.sum() <= 3
