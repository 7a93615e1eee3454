"""Mainlobe width (Sec. 5.1) and var(|s|) (Eq. 22) through the C ABI against
the FP64 reference."""
import numpy as np
import pytest

from oracle import composite
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


@pytest.mark.parametrize("N", [4, 13, 64, 300, 1024])
@pytest.mark.parametrize("kind", ["phase", "complex"])
@pytest.mark.parametrize("gamma", [8.0, 50.0])
def test_width_and_modulus_terms_match_reference(N, kind, gamma):
    B = 5
    if kind == "phase":
        ph = inputs.random_phases(91 + N, B, N)
        x = torch.from_numpy(ph).to(_dev())
        sigs = [np.exp(1j * ph[b].astype(np.float64)) for b in range(B)]
    else:
        # a mean offset puts some lags near the -3 dB threshold (non-flat gradient)
        z = (inputs.random_complex(92 + N, B, N) + 0.7).astype(np.complex64)
        x = torch.from_numpy(z).to(_dev())
        sigs = [z[b].astype(np.complex128) for b in range(B)]
    wW, wV = 0.3, 2.0
    terms, grad = g.composite_terms(x, gamma, 1e-12, wW, wV)
    terms, grad = terms.cpu().numpy(), grad.cpu().numpy()
    for b in range(B):
        W, gsW, gpW = composite.mainlobe_width_grad(sigs[b], gamma, 1e-12)
        V, gsV = composite.modulus_variance_grad(sigs[b])
        assert abs(terms[b, 0] - W) <= 1e-4 * max(W, 1.0), (b, terms[b, 0], W)
        assert abs(terms[b, 1] - V) <= 1e-5 * max(V, 1e-3)
        ref = wW * gpW if kind == "phase" else wW * gsW + wV * gsV
        nr = np.linalg.norm(ref)
        if nr < 1e-6:
            assert np.linalg.norm(grad[b]) <= 1e-5
        else:
            assert np.linalg.norm(grad[b] - ref) <= 1e-3 * nr, (b, np.linalg.norm(grad[b] - ref) / nr)


def test_rect_pulse_width_on_gpu():
    N = 64
    x = torch.ones((1, N), dtype=torch.complex64, device=_dev())
    terms, _ = g.composite_terms(x, 50.0, 0.0, 1.0, 0.0)
    assert abs(float(terms[0, 0]) - composite.mainlobe_width(np.ones(N), 50.0)) < 1e-3
