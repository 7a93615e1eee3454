"""The target-matching term (L_match of Eq. 22) through the C ABI against the
FP64 reference: loss, phase and complex gradients, accumulation."""
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


def _lfm_target(N, M, w):
    """A thumb-tack-free reference: the surface of a discrete LFM chirp."""
    s = np.exp(1j * np.pi * np.arange(N) ** 2 / N)
    return oracle.af_ahat(s, M, w[0], w[1], w[2], w[3], 1e-12) ** 2


CASES = [
    (16, 64, (-15, 15, -32, 31, -1, -1)),
    (48, 128, (-20, 30, -40, 50, -1, -1)),
    (100, 256, (-99, 99, -128, 127, -1, -1)),
    (300, 512, (5, 120, -64, 64, -1, -1)),
]


@pytest.mark.parametrize("N,M,w", CASES)
@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_match_matches_oracle(N, M, w, kind):
    B = 3
    tgt = _lfm_target(N, M, w)
    target = torch.from_numpy(np.broadcast_to(tgt, (B,) + tgt.shape).astype(np.float32).copy()).to(_dev())
    if kind == "phase":
        ph = inputs.random_phases(111 + N, B, N)
        x = torch.from_numpy(ph).to(_dev())
        sigs = [np.exp(1j * ph[b].astype(np.float64)) for b in range(B)]
    else:
        z = inputs.random_complex(112 + N, B, N)
        x = torch.from_numpy(z).to(_dev())
        sigs = [z[b].astype(np.complex128) for b in range(B)]
    loss, grad = g.af_match(x, M, g.Window(*w), target, 0.8)
    loss, grad = loss.cpu().numpy(), grad.cpu().numpy()
    for b in range(B):
        rl, rgs, rgp = oracle.match(sigs[b], M, w, target[b].cpu().numpy().astype(np.float64), 0.8)
        assert abs(loss[b] - rl) <= 1e-4 * rl, (b, loss[b], rl)
        ref = rgp if kind == "phase" else rgs
        assert np.linalg.norm(grad[b] - ref) <= 1e-4 * np.linalg.norm(ref), (b, np.linalg.norm(grad[b] - ref) / np.linalg.norm(ref))


def test_match_accumulates():
    N, M = 64, 128
    w = g.Window.full(N, M, k_ml=-1, m_ml=-1)
    tgt = torch.zeros((2, 2 * N - 1, M), device=_dev())
    x = torch.from_numpy(inputs.random_phases(121, 2, N)).to(_dev())
    _, g1 = g.af_match(x, M, w, tgt, 1.0)
    base = torch.from_numpy(inputs.random_phases(122, 2, N)).to(_dev())
    acc = base.clone()
    nb = g.graf_af_match_workspace_bytes(2, N, M, w.c())
    ws = torch.empty(nb, dtype=torch.uint8, device=_dev())
    out8 = torch.ones((2, 8), device=_dev())
    loss = torch.empty(2, device=_dev())
    st = g.graf_af_match(x.data_ptr(), g.GRAF_IN_PHASE, 2, N, M, w.c(), tgt.data_ptr(), 1.0, 1e-12, loss.data_ptr(),
                         out8.data_ptr(), None, acc.data_ptr(), 1, ws.data_ptr(), nb,
                         torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    assert torch.allclose(acc, base + g1, rtol=1e-5, atol=1e-7)
    assert torch.allclose(out8[:, 0], 1.0 + loss, rtol=1e-6)
