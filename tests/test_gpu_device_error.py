"""The device error word: the loss finalisation raises a bit for a waveform
whose energy is zero or not finite and for a non-finite loss, and
graf_get_device_error takes (reads and clears) it in stream order.  The bad
inputs only give NaN or Inf in floating point: no index depends on a value."""
import numpy as np
import pytest

from paper_2506_22935_gb300 import _build, inputs
from paper_2506_22935_gb300 import graf as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    g.load()


def _dev():
    return torch.device("cuda:0")


def _stream():
    return torch.cuda.current_stream(_dev()).cuda_stream


def test_clean_calls_raise_nothing():
    g.device_error_word()  # start from a clear word
    N, M = 64, 128
    x = torch.from_numpy(inputs.random_phases(81, 3, N)).to(_dev())
    g.af_loss_backward(x, M, g.Window.full(N, M), g.Loss())
    assert g.device_error_word() == 0
    assert g.graf_get_device_error(_stream()) == g.GRAF_OK


def test_zero_energy_waveform_raises_and_clears():
    g.device_error_word()
    N, M = 64, 128
    z = inputs.random_complex(82, 3, N)
    z[1] = 0.0  # E = 0: the normalisation is undefined
    x = torch.from_numpy(z).to(_dev())
    w, loss = g.Window.full(N, M), g.Loss()
    out8 = torch.empty((3, 8), dtype=torch.float32, device=_dev())
    nb = g.graf_af_loss_workspace_bytes(3, N, M, w.c())
    ws = torch.empty(nb, dtype=torch.uint8, device=_dev())
    st = g.graf_af_loss(x.data_ptr(), g.GRAF_IN_COMPLEX, 3, N, M, w.c(), loss.c(), out8.data_ptr(),
                        ws.data_ptr(), nb, _stream())
    assert st == g.GRAF_OK  # the call itself cannot see the values
    word = g.device_error_word()
    assert word & g.GRAF_DEVERR_ENERGY
    assert g.device_error_word() == 0  # taken
    o = out8.cpu().numpy()
    assert np.all(np.isfinite(o[[0, 2], 0]))


def test_nan_phase_raises_nonfinite_through_status():
    g.device_error_word()
    N, M = 32, 64
    ph = inputs.random_phases(83, 2, N)
    ph[0, 5] = np.nan
    x = torch.from_numpy(ph).to(_dev())
    g.af_loss_backward(x, M, g.Window.full(N, M), g.Loss())
    assert g.graf_get_device_error(_stream()) == g.GRAF_ERR_DEVICE_FLAG
    assert g.graf_get_device_error(_stream()) == g.GRAF_OK
