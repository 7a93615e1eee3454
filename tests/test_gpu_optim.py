"""On-device optimiser (Adam on phases, captured in a CUDA graph) against the
FP64 oracle's optimiser."""
import time

import numpy as np
import pytest

import oracle as orc
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


def test_adam_kernel_matches_oracle():
    rng = np.random.default_rng(11)
    n = 1000
    x0 = rng.standard_normal(n).astype(np.float32)
    x = torch.from_numpy(x0.copy()).to(_dev())
    m = torch.zeros_like(x)
    v = torch.zeros_like(x)
    step = torch.zeros(1, dtype=torch.int32, device=_dev())
    state = torch.zeros(g.graf_adam_state_bytes(), dtype=torch.uint8, device=_dev())
    hp = g.graf_adam_t(0.01, 0.9, 0.999, 1e-8)
    xr, mr, vr = x0.astype(np.float64), np.zeros(n), np.zeros(n)
    st = torch.cuda.current_stream().cuda_stream
    for t in range(1, 7):
        gr = (rng.standard_normal(n) * t).astype(np.float32)
        gd = torch.from_numpy(gr).to(_dev())
        assert g.graf_adam_step(x.data_ptr(), m.data_ptr(), v.data_ptr(), gd.data_ptr(), n, hp, step.data_ptr(),
                                state.data_ptr(), st) == 0
        xr, mr, vr = orc.adam_update(xr, mr, vr, gr.astype(np.float64), t)
    torch.cuda.synchronize()
    assert int(step.item()) == 6
    assert int(state.view(torch.int32)[0].item()) == 0
    np.testing.assert_allclose(x.cpu().numpy(), xr, rtol=0, atol=2e-6)
    np.testing.assert_allclose(m.cpu().numpy(), mr, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("win,lp", [
    ((-10, 10, -20, 20, 0, 0), (0.0, 1.0, 50.0)),   # masked ISL
    (None, (1.0, 1.0, 50.0)),                       # full AF, PSL + ISL
])
def test_optimiser_matches_oracle(win, lp):
    from paper_2506_22935_gb300.optim import Adam, PhaseOptimizer
    B, N, M, steps = 2, 48, 128, 10
    phi0 = inputs.random_phases(31, B, N)
    w = g.Window.full(N, M) if win is None else g.Window(*win)
    loss = g.Loss(lp[0], lp[1], lp[2], 1e-12)
    phi = torch.from_numpy(phi0.copy()).to(_dev())
    opt = PhaseOptimizer(phi, M, w, loss, Adam(lr=0.01), history_len=steps)
    opt.run(steps, graph=True)
    torch.cuda.synchronize()
    got_phi = phi.cpu().numpy()
    got_hist = opt.history.cpu().numpy()
    for b in range(B):
        ref_phi, ref_hist = orc.optimize_phases(phi0[b].astype(np.float64), M, w.as_tuple(), loss.w_psl, loss.w_isl,
                                                loss.beta, loss.eps, steps, lr=0.01)
        np.testing.assert_allclose(got_hist[:, b], ref_hist, rtol=1e-4)
        np.testing.assert_allclose(got_phi[b], ref_phi, rtol=0, atol=1e-3)


def test_graph_replay_equals_eager_steps():
    from paper_2506_22935_gb300.optim import PhaseOptimizer
    B, N, M, steps = 3, 200, 512, 12
    phi0 = torch.from_numpy(inputs.random_phases(41, B, N)).to(_dev())
    w, loss = g.Window.masked(60, 100), g.Loss(0.0, 1.0, 50.0, 1e-12)
    a = PhaseOptimizer(phi0.clone(), M, w, loss, history_len=steps)
    b = PhaseOptimizer(phi0.clone(), M, w, loss, history_len=steps)
    a.run(steps, graph=False)
    b.run(steps, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a.phi, b.phi)
    assert torch.equal(a.history, b.history)
    # replaying the same graph continues from the current state
    b.reset(phi0)
    b.run(steps, graph=True)
    torch.cuda.synchronize()
    assert torch.equal(a.phi, b.phi)


def test_masked_isl_workload_64x4096_m8192_500_steps():
    """64 random-phase codes, N = 4096, M = 8192, mask |k| <= 512, |m| <= 256
    minus the origin, masked ISL, 500 Adam steps (lr 1e-2) in one captured
    CUDA graph.  The first step's loss and gradient of code 0 are checked
    against the oracle; every code's masked ISL must fall."""
    from paper_2506_22935_gb300.optim import Adam, PhaseOptimizer
    B, N, M, steps = 64, 4096, 8192, 500
    phi0 = inputs.random_phases(inputs.SEED_BASE + 3, B, N)
    w, loss = g.Window.masked(512, 256), g.Loss(0.0, 1.0, 50.0, 1e-12)
    x = torch.from_numpy(phi0.copy()).to(_dev())
    out8, grad = g.af_loss_backward(x[:1], M, w, loss)
    _, rp, o8 = orc.grad(orc.signal_from_phase(phi0[0].astype(np.float64)), M, w.as_tuple(), 0.0, 1.0, 50.0, 1e-12)
    assert abs(out8[0, 0].item() - o8[0]) <= 1e-5 * o8[0]
    gd = grad[0].cpu().numpy()
    assert np.linalg.norm(gd - rp) / np.linalg.norm(rp) <= 1e-4
    opt = PhaseOptimizer(x, M, w, loss, Adam(lr=1e-2), history_len=steps)
    graph = opt.capture(steps)
    opt.reset(torch.from_numpy(phi0).to(_dev()))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    graph.replay()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h = opt.history.cpu().numpy()
    assert np.all(np.isfinite(h))
    assert abs(h[0, 0] - o8[0]) <= 1e-5 * o8[0]
    assert np.all(h[-1] < 0.9 * h[0])
    print(f"500 steps in {dt:.3f} s, masked ISL {h[0].mean():.2f} -> {h[-1].mean():.2f}")
