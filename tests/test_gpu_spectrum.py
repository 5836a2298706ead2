"""Cyclic spectra on the GPU (cyc_read_spectrum) against the oracle's spectrum of the
oracle's estimate: rectangular and Hann lag windows, signed lags, two inputs, Full mode,
host and device outputs.  Error metric: max |S_gpu - S_oracle| over R^0(0) sum_l w(m_l)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def push_all(s, x, y=None):
    import torch
    xt = torch.from_numpy(x.view(np.float32).copy()).cuda()
    if y is None:
        s.push(xt)
    else:
        s.push(xt, y=torch.from_numpy(y.view(np.float32).copy()).cuda())


@pytest.mark.parametrize("taper", [0, 1])
@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16x3", 1e-4)])
def test_spectrum_one_input(cyc, taper, precision, tol):
    T = 8000
    x = (synth.gmsk(T, bt=0.3, sps=8, seed=5) * np.exp(2j * np.pi * 0.05 * np.arange(T))).astype(np.complex64)
    lags = np.arange(-16, 17)
    alphas = np.array([0.0, 0.125, 0.1625, -0.3])
    with cyc.Stream(lags, alphas, 3, precision=precision) as s:
        push_all(s, x)
        S = s.read_spectrum(64, taper)
        R, _ = s.read()
    Ro, _ = oracle.estimate_xy(x, None, lags, alphas)
    So = oracle.spectrum(Ro, lags, 64, taper)
    scale = oracle.r00_xy(x, None, 16, 16) * np.sum(oracle.lag_window(lags, taper))
    assert np.max(np.abs(S - So)) / scale < tol
    # the spectrum of the GPU estimate is the DFT of what cyc_read returns
    assert np.max(np.abs(S - oracle.spectrum(R, lags, 64, taper))) / scale < 1e-12


def test_spectrum_two_inputs_full_mode_device_output(cyc):
    import torch
    T, A = 6000, 128
    x = synth.white(T, seed=180).astype(np.complex64)
    y = (np.roll(x, 4) * np.exp(2j * np.pi * 0.2 * np.arange(T))).astype(np.complex64)
    lags = np.array([-6, -2, 0, 3, 4, 9])
    with cyc.Stream(lags, None, 3, cross=True, full=A) as s:
        push_all(s, x, y)
        out = torch.empty((2, A, 40, 2), dtype=torch.float64, device="cuda")
        s.read_spectrum(40, 1, out)
        S = out.cpu().numpy()
    S = S[..., 0] + 1j * S[..., 1]
    Ro, _ = oracle.estimate_xy(x, y, lags, -0.5 + np.arange(A) / A)
    So = oracle.spectrum(Ro, lags, 40, 1)
    scale = oracle.r00_xy(x, y, 6, 9) * np.sum(oracle.lag_window(lags, 1))
    assert np.max(np.abs(S - So)) / scale < 1e-5


def test_spectrum_errors(cyc):
    with cyc.Stream([0, 1], [0.1], 3) as s:
        with pytest.raises(cyc.CycError) as e:
            s.read_spectrum(8)
        assert e.value.code == cyc.CYC_ENODATA
        push_all(s, synth.white(100, seed=1).astype(np.complex64))
        for Q, taper in ((0, 0), (8, 2)):
            with pytest.raises(cyc.CycError) as e:
                s.read_spectrum(Q, taper)
            assert e.value.code == cyc.CYC_EINVAL
