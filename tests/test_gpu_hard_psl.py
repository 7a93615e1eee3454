"""The hard PSL of Eq. 18 (the loss's beta = +inf: the maximum of Ahat^2 over
Omega, with the subgradient through one arg-max cell) through the C ABI,
against the FP64 oracle: loss scalars, and gradients of the aperiodic and
periodic AF, alone and with ISL, phase and complex input.

Where two cells are maximal within FP32 rounding, either is a correct
arg-max: the GPU gradient is checked against the oracle's gradient through
each cell whose FP64 Ahat^2 lies within a relative 1e-5 of the maximum (the
loss value itself is unique)."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2506_22935_gb300 import _build, inputs
from paper_2506_22935_gb300 import graf as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

INF = math.inf
G_TOL = 1e-4
L_TOL = 1e-5
NEAR = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    g.load()


def _dev():
    return torch.device("cuda:0")


def _rel(a, b):
    """Relative L2 error, with an absolute floor of 1e-7 (a peak on row 0 of a
    phase code, with the ISL of whole rows, has an exactly zero gradient,
    which both sides give as rounding noise: ~1e-20 in FP64, ~1e-13 in FP32)."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-7))


def _candidates(A2, win):
    """Cells (k, m) of Omega whose Ahat^2 is within NEAR of the maximum."""
    ks = np.arange(win[0], win[1] + 1)[:, None]
    ms = np.arange(win[2], win[3] + 1)[None, :]
    omega = ~((np.abs(ks) <= win[4]) & (np.abs(ms) <= win[5]))
    A = np.where(omega, A2, -np.inf)
    top = A.max()
    idx = np.argwhere(A >= top * (1 - NEAR))
    return [(int(win[0] + i), int(win[2] + j)) for i, j in idx]


def _check_grad(got, want_isl, cell_grads, what):
    """got must equal the ISL part plus one candidate cell's gradient."""
    errs = [_rel(got, want_isl + c) for c in cell_grads]
    assert min(errs) <= G_TOL, (what, errs)


def _signals(kind, seed, B, N):
    if kind == "phase":
        ph = inputs.random_phases(seed, B, N)
        return torch.from_numpy(ph).to(_dev()), [orc.signal_from_phase(ph[b].astype(np.float64)) for b in range(B)]
    z = inputs.random_complex(seed, B, N)
    return torch.from_numpy(z).to(_dev()), [z[b].astype(np.complex128) for b in range(B)]


CASES = [
    # N, M, window (None: whole AF minus the zero-delay mainlobe)
    (64, 128, None),
    (100, 256, (-60, 45, -128, 127, 0, 2)),
    (300, 512, (-299, 299, -40, 90, 0, 3)),
    (200, 256, (5, 150, -128, 127, -1, -1)),
    (1024, 2048, None),
]


@pytest.mark.parametrize("N,M,win", CASES)
@pytest.mark.parametrize("kind", ["phase", "complex"])
@pytest.mark.parametrize("w_isl", [0.0, 0.5])
def test_hard_psl_loss_and_gradient(N, M, win, kind, w_isl):
    B = 3 if N < 1024 else 1
    win = win or orc.full_window(N, M)
    w = g.Window(*win)
    loss = g.Loss(1.0, w_isl, INF, 1e-12)
    x, sigs = _signals(kind, 700 + N, B, N)
    out8, grad = g.af_loss_backward(x, M, w, loss)
    only8 = g.af_loss(x, M, w, loss)
    gsep = g.af_backward(x, M, w, loss, only8)
    torch.cuda.synchronize()
    out8, only8 = out8.cpu().numpy(), only8.cpu().numpy()
    grad, gsep = grad.cpu().numpy(), gsep.cpu().numpy()
    for b in range(B):
        s = sigs[b]
        gs_isl, gp_isl, o8 = orc.grad(s, M, win, 0.0, w_isl, INF, 1e-12)
        # the oracle's scalars of the hard loss: L = PSL_hard + w_isl ISL,
        # PSL = S_p = PSL_hard
        ref8 = [o8[3] + w_isl * o8[2], o8[3], o8[2], o8[3], o8[4], o8[5], o8[3]]
        for i in (0, 1, 2, 3, 6):
            assert abs(out8[b, i] - ref8[i]) <= L_TOL * max(abs(ref8[i]), 1e-6), (b, i, out8[b], ref8)
            assert abs(only8[b, i] - ref8[i]) <= L_TOL * max(abs(ref8[i]), 1e-6), (b, i, only8[b], ref8)
        assert out8[b, 5] == np.float32(ref8[5])
        A2 = orc.af_ahat(s, M, win[0], win[1], win[2], win[3], 1e-12) ** 2
        cands = _candidates(A2, win)
        cg = [orc.cell_grad(s, M, k, m, 1e-12)[0 if kind == "complex" else 1] for k, m in cands]
        want = gs_isl if kind == "complex" else gp_isl
        _check_grad(grad[b], want, cg, ("fused", b, cands))
        _check_grad(gsep[b], want, cg, ("separate backward", b, cands))


@pytest.mark.parametrize("N", [16, 64, 256])
@pytest.mark.parametrize("sign", [1, -1])
@pytest.mark.parametrize("kind", ["phase", "complex"])
@pytest.mark.parametrize("w_isl", [0.0, 0.25])
def test_periodic_hard_psl(N, sign, kind, w_isl):
    B = 3
    win = orc.full_pwindow(N)
    loss = g.Loss(1.0, w_isl, INF, 1e-12)
    x, sigs = _signals(kind, 900 + N, B, N)
    out8, grad = g.paf_loss_backward(x, g.Window(*win), loss, sign)
    torch.cuda.synchronize()
    out8, grad = out8.cpu().numpy(), grad.cpu().numpy()
    for b in range(B):
        s = sigs[b]
        gs_isl, gp_isl, _ = orc.pgrad(s, win, 0.0, w_isl, INF, 1e-12, sign=sign)
        ref8 = orc.ploss(s, win, 1.0, w_isl, INF, 1e-12, sign=sign)
        for i in (0, 1, 2, 3):
            assert abs(out8[b, i] - ref8[i]) <= L_TOL * max(abs(ref8[i]), 1e-6), (b, i, out8[b], ref8)
        A2 = np.abs(orc.paf_complex(s, sign)) ** 2 / orc.energy(s) ** 2
        cands = _candidates(A2, win)
        cg = [orc.pcell_grad(s, k, m, 1e-12, sign=sign)[0 if kind == "complex" else 1] for k, m in cands]
        want = gs_isl if kind == "complex" else gp_isl
        _check_grad(grad[b], want, cg, (b, cands))


def test_hard_psl_upstream_scaling_and_autograd():
    N, M, B = 128, 256, 4
    w = g.Window.full(N, M)
    loss = g.Loss(0.7, 0.0, INF, 1e-12)
    x = torch.from_numpy(inputs.random_phases(1234, B, N)).to(_dev())
    dL = torch.tensor([1.0, -2.0, 0.5, 3.0], device=_dev())
    _, g1 = g.af_loss_backward(x, M, w, loss)
    _, g2 = g.af_loss_backward(x, M, w, loss, dL=dL)
    torch.cuda.synchronize()
    assert torch.allclose(g2, g1 * dL[:, None], rtol=1e-6, atol=1e-9)
    xr = x.clone().requires_grad_(True)
    L, _ = g.af_loss_autograd(xr, M, w, loss)
    (L * dL).sum().backward()
    torch.cuda.synchronize()
    assert torch.allclose(xr.grad, g2, rtol=1e-6, atol=1e-9)


def test_hard_psl_empty_omega():
    """A window that the mainlobe box covers: every scalar 0, gradient 0."""
    N, M = 32, 64
    w = g.Window(-2, 2, -3, 3, 5, 5)
    x = torch.from_numpy(inputs.random_phases(5, 2, N)).to(_dev())
    out8, grad = g.af_loss_backward(x, M, w, g.Loss(1.0, 0.0, INF, 1e-12))
    torch.cuda.synchronize()
    assert torch.all(out8[:, [0, 1, 2, 3, 6]] == 0) and torch.all(grad == 0)
    assert torch.all(out8[:, 5] == 0)


def test_soft_psl_above_the_fixed_shift_limit():
    """beta above the fixed log-sum-exp shift's range (beta log2(e) / 2 > 88)
    runs the running-maximum form: loss and gradient against the oracle."""
    N, M, B = 128, 256, 2
    win = orc.full_window(N, M)
    loss = g.Loss(1.0, 0.5, 400.0, 1e-12)
    ph = inputs.random_phases(66, B, N)
    out8, grad = g.af_loss_backward(torch.from_numpy(ph).to(_dev()), M, g.Window(*win), loss)
    torch.cuda.synchronize()
    for b in range(B):
        _, gp, ref8 = orc.grad(orc.signal_from_phase(ph[b].astype(np.float64)), M, win, 1.0, 0.5, 400.0, 1e-12)
        for i in (0, 1, 2, 3):
            assert abs(float(out8[b, i]) - ref8[i]) <= L_TOL * abs(ref8[i])
        assert _rel(grad[b].cpu().numpy(), gp) <= G_TOL
