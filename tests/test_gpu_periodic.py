"""The periodic AF of the paper's own definition (Eq. 7, Algorithm 1) through
the C ABI against the FP64 periodic oracle: chi, loss scalars and gradients,
both exponent signs, phase and complex input."""
import math

import numpy as np
import pytest

import oracle
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


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-30))


@pytest.mark.parametrize("N", [8, 16, 64, 256, 2048])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_periodic_chi_matches_oracle(N, sign, kind):
    B = 2
    if kind == "phase":
        ph = inputs.random_phases(31 + N, B, N)
        x = torch.from_numpy(ph).to(_dev())
        sigs = [np.exp(1j * ph[b].astype(np.float64)) for b in range(B)]
    else:
        z = inputs.random_complex(32 + N, B, N)
        x = torch.from_numpy(z).to(_dev())
        sigs = [z[b].astype(np.complex128) for b in range(B)]
    chi = g.paf_forward(x, sign, normalise=True).cpu().numpy()
    chi_raw = g.paf_forward(x, sign, normalise=False).cpu().numpy()
    for b in range(B):
        if N <= 256:
            ref = oracle.paf_chi(sigs[b], sign, normalise=True)
            assert np.abs(chi[b] - ref).max() <= 2e-5
            raw = oracle.paf_chi(sigs[b], sign, normalise=False)
            assert np.abs(chi_raw[b] - raw).max() <= 2e-5 * raw.max()
        else:
            # sampled cells, each its own FP64 direct sum
            rng = np.random.default_rng(N + b)
            for _ in range(24):
                k, m = (int(v) for v in rng.integers(-(N // 2), N // 2, size=2))
                X = oracle.paf_complex(sigs[b], sign, k, k, m, m)[0, 0]
                ref = abs(X) ** 2 / oracle.energy(sigs[b]) ** 2
                assert abs(chi[b, k + N // 2, m + N // 2] - ref) <= 2e-5


@pytest.mark.parametrize("sign", [1, -1])
def test_chu_ridge_on_gpu(sign):
    N, u = 256, 5
    n = np.arange(N, dtype=np.float64)
    ph = (-(math.pi * u * n * n / N) % (2 * math.pi)).astype(np.float32)
    chi = g.paf_forward(torch.from_numpy(ph[None]).to(_dev()), sign, normalise=True)[0].cpu().numpy()
    k = np.arange(-(N // 2), N // 2)[:, None]
    m = np.arange(-(N // 2), N // 2)[None, :]
    on = ((m - sign * u * k) % N) == 0
    assert np.abs(chi[on] - 1.0).max() <= 1e-4
    assert chi[~on].max() <= 1e-6


WINDOWS = [
    ("full", lambda N: (-(N // 2), N // 2 - 1, -(N // 2), N // 2 - 1, 0, 0)),
    ("box", lambda N: (-(N // 2), N // 2 - 1, -(N // 2), N // 2 - 1, 1, 1)),
    ("masked", lambda N: (-(N // 8), N // 8, -(N // 16), N // 16, 0, 0)),
    ("kpos", lambda N: (1, N // 4, -(N // 2), N // 2 - 1, -1, -1)),
]
LOSSES = [(1.0, 1.0, 50.0), (0.0, 1.0, 50.0), (1.0, 0.0, 20.0)]


@pytest.mark.parametrize("wname,wf", WINDOWS)
@pytest.mark.parametrize("lp", LOSSES)
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_periodic_loss_and_gradient_match_oracle(wname, wf, lp, sign, kind):
    N, B = 64, 3
    win = wf(N)
    if kind == "phase":
        ph = inputs.random_phases(41, B, N)
        x = torch.from_numpy(ph).to(_dev())
        sigs = [np.exp(1j * ph[b].astype(np.float64)) for b in range(B)]
    else:
        z = inputs.random_complex(42, B, N)
        x = torch.from_numpy(z).to(_dev())
        sigs = [z[b].astype(np.complex128) for b in range(B)]
    out8, grad = g.paf_loss_backward(x, g.Window(*win), g.Loss(lp[0], lp[1], lp[2], 1e-12), sign)
    out8, grad = out8.cpu().numpy(), grad.cpu().numpy()
    for b in range(B):
        gs, gp, o = oracle.pgrad(sigs[b], win, lp[0], lp[1], lp[2], 1e-12, sign)
        for i in (0, 1, 2, 3, 4, 5):
            assert abs(out8[b, i] - o[i]) <= 1e-5 * max(abs(o[i]), 1e-3), (i, out8[b, i], o[i])
        ref = gp if kind == "phase" else gs
        scale = np.linalg.norm(ref)
        if scale < 1e-9:   # a full-window ISL has an exactly zero phase gradient
            assert np.linalg.norm(grad[b]) <= 1e-6
        else:
            assert _rel(grad[b], ref) <= 1e-4, (b, _rel(grad[b], ref))


def test_periodic_full_size_loss_matches_oracle():
    """N = 1024 (the paper's experiments use N = 256): loss scalars of two
    codes against the FP64 oracle, the gradient against global-phase
    invariance and the oracle gradient of the first."""
    N, B = 1024, 2
    ph = inputs.random_phases(51, B, N)
    x = torch.from_numpy(ph).to(_dev())
    win = g.Window.periodic(N)
    out8, grad = g.paf_loss_backward(x, win, g.Loss(1.0, 1.0, 50.0, 1e-12), 1)
    out8, grad = out8.cpu().numpy(), grad.cpu().numpy()
    s0 = np.exp(1j * ph[0].astype(np.float64))
    o = oracle.ploss(s0, win.as_tuple(), 1.0, 1.0, 50.0, 1e-12, 1)
    assert abs(out8[0, 0] - o[0]) <= 1e-5 * abs(o[0])
    assert abs(out8[0, 3] - o[3]) <= 1e-5 * abs(o[3])
    for b in range(B):
        assert abs(grad[b].sum()) <= 1e-3 * np.abs(grad[b]).sum()
