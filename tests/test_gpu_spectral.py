"""Spectral variance (the LPI term of Eq. 25) and its gradient through the C
ABI against the FP64 reference; accumulation into an AF gradient and the loss
record."""
import numpy as np
import pytest

from oracle import spectral
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


def _ref(sig):
    """FP64 reference: the direct-DFT oracle for small N; for large N the same
    formulas with numpy's FFT (a library routine) for the two transforms."""
    N = sig.shape[0]
    if N <= 1024:
        return spectral.spectral_variance_grad(sig)
    S = np.fft.fft(sig)
    P = np.abs(S) ** 2
    q = P / P.sum()
    sv = np.mean((q - 1.0 / N) ** 2)
    dq = (2.0 / N) * (q - 1.0 / N)
    dP = (dq - np.sum(q * dq)) / P.sum()
    gr = np.fft.ifft(dP * S) * N
    return sv, 2.0 * gr, 2.0 * np.imag(gr * np.conj(sig))


@pytest.mark.parametrize("N", [8, 64, 256, 2048, 16384])
@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_spectral_variance_matches_reference(N, kind):
    B = 37 if N <= 2048 else 3  # not a multiple of the slots per CTA
    if kind == "phase":
        ph = inputs.random_phases(61 + N, B, N)
        x = torch.from_numpy(ph).to(_dev())
        sigs = [np.exp(1j * ph[b].astype(np.float64)) for b in range(B)]
    else:
        z = inputs.random_complex(62 + N, B, N)
        x = torch.from_numpy(z).to(_dev())
        sigs = [z[b].astype(np.complex128) for b in range(B)]
    w = 2000.0
    sv, grad = g.spectral_variance(x, w)
    sv, grad = sv.cpu().numpy(), grad.cpu().numpy()
    for b in range(B):
        rs, rgs, rgp = _ref(sigs[b])
        assert abs(sv[b] - rs) <= 1e-4 * rs, (b, sv[b], rs)
        ref = w * (rgp if kind == "phase" else rgs)
        assert np.linalg.norm(grad[b] - ref) <= 1e-4 * np.linalg.norm(ref), b


def test_accumulates_into_gradient_and_loss_record():
    B, N = 5, 256
    ph = inputs.random_phases(71, B, N)
    x = torch.from_numpy(ph).to(_dev())
    base = torch.from_numpy(inputs.random_phases(72, B, N)).to(_dev())
    grad = base.clone()
    out8 = torch.ones((B, 8), dtype=torch.float32, device=_dev())
    st = g.graf_spectral_variance(x.data_ptr(), g.GRAF_IN_PHASE, B, N, 7.0, out8.data_ptr(), None, None,
                                  grad.data_ptr(), 1, torch.cuda.current_stream().cuda_stream)
    assert st == 0
    sv, g1 = g.spectral_variance(x, 7.0)
    torch.cuda.synchronize()
    assert torch.allclose(grad, base + g1, rtol=1e-6, atol=1e-7)
    assert torch.allclose(out8[:, 0], 1.0 + 7.0 * sv, rtol=1e-6)
    assert torch.equal(out8[:, 7], sv)
    assert torch.equal(out8[:, 1:7], torch.ones((B, 6), device=_dev()))


def test_flat_spectrum_has_zero_variance_and_gradient():
    N = 1024
    n = np.arange(N, dtype=np.float64)
    ph = (-(np.pi * n * n / N) % (2 * np.pi)).astype(np.float32)  # a Chu sequence
    sv, grad = g.spectral_variance(torch.from_numpy(ph[None]).to(_dev()), 1.0)
    assert float(sv[0]) < 1e-10
    assert float(grad.abs().max()) < 1e-6
