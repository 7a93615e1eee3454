"""Ragged batches (graf_batch_*): waveforms of unequal length, each with its
own Doppler length, window and loss, in persistent per-M launches; parity with
the FP64 oracle per waveform."""
import numpy as np
import pytest

import oracle as orc
from paper_2506_22935_gb300 import _build, inputs
from paper_2506_22935_gb300 import graf as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G_TOL = 1e-4
L_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    g.load()


def _dev():
    return torch.device("cuda:0")


def _packed_phases(seed, Ns):
    phis = [inputs.random_phases(seed + i, 1, int(n))[0] for i, n in enumerate(Ns)]
    return phis, np.concatenate(phis)


def _check(plan, phis, out8, grad, windows, losses, Ms):
    out8 = out8.cpu().numpy()
    grad = grad.cpu().numpy()
    for b, phi in enumerate(phis):
        N, M = len(phi), Ms[b]
        w = windows[b]
        l = losses[b] if len(losses) > 1 else losses[0]
        s = orc.signal_from_phase(phi.astype(np.float64))
        _, gp, o8 = orc.grad(s, M, w.as_tuple(), l.w_psl, l.w_isl, l.beta, l.eps)
        for i in (0, 1, 2, 3):
            assert abs(out8[b, i] - o8[i]) <= L_TOL * max(abs(o8[i]), 1e-6), (b, i, out8[b], o8)
        assert out8[b, 5] == np.float32(o8[5])
        gb = grad[plan.offsets[b]:plan.offsets[b + 1]]
        if np.linalg.norm(gp) < 1e-9:
            assert np.abs(gb).max() < 1e-6
        else:
            rel = np.linalg.norm(gb - gp) / np.linalg.norm(gp)
            assert rel <= G_TOL, (b, N, M, rel)


def test_ragged_batch_default_windows_matches_oracle():
    Ns = [20, 33, 64, 100, 129, 200, 255, 256, 300, 47, 90, 150]
    phis, packed = _packed_phases(70, Ns)
    loss = g.Loss(1.0, 1.0, 50.0, 1e-12)
    plan = g.BatchPlan(Ns, losses=[loss])
    Ms = [1 << int(np.ceil(np.log2(2 * n))) for n in Ns]
    windows = [g.Window.full(n, m) for n, m in zip(Ns, Ms)]
    info = plan.info()
    assert sorted(b["M"] for b in info) == sorted(set(Ms))
    assert all(b["fused"] for b in info)
    out8, grad = plan.loss_backward(torch.from_numpy(packed).to(_dev()))
    torch.cuda.synchronize()
    _check(plan, phis, out8, grad, windows, [loss], Ms)


def test_ragged_batch_per_waveform_windows_and_losses():
    """Masked windows with PSL run the loss kernel then the recomputing
    backward; ISL-only and full-window waveforms share buckets with them."""
    Ns = [40, 64, 100, 128, 180, 250, 31, 77]
    Ms = [128, 128, 256, 256, 512, 512, 64, 256]
    windows = [g.Window.masked(10, 20), g.Window.full(64, 128), g.Window(-30, 12, -64, 100, 0, 0),
               g.Window.masked(60, 40), g.Window.full(180, 512), g.Window(5, 200, -256, 255, -1, -1),
               g.Window.full(31, 64), g.Window.masked(30, 127)]
    losses = [g.Loss(1.0, 1.0, 50.0, 1e-12), g.Loss(0.0, 1.0, 50.0, 1e-12), g.Loss(0.5, 2.0, 20.0, 1e-12),
              g.Loss(0.0, 1.0, 50.0, 1e-12), g.Loss(1.0, 0.0, 50.0, 1e-12), g.Loss(1.0, 1.0, 10.0, 1e-12),
              g.Loss(2.0, 1.0, 80.0, 1e-12), g.Loss(1.0, 1.0, 50.0, 1e-12)]
    phis, packed = _packed_phases(90, Ns)
    plan = g.BatchPlan(Ns, M=Ms, windows=windows, losses=losses)
    info = plan.info()
    assert any(not b["fused"] for b in info)
    out8, grad = plan.loss_backward(torch.from_numpy(packed).to(_dev()))
    torch.cuda.synchronize()
    _check(plan, phis, out8, grad, windows, losses, Ms)


def test_ragged_batch_equals_uniform_calls_and_autotune():
    Ns = [300, 250, 300, 120, 300, 64]
    phis, packed = _packed_phases(120, Ns)
    loss = g.Loss(1.0, 1.0, 50.0, 1e-12)
    plan = g.BatchPlan(Ns, losses=[loss])
    x = torch.from_numpy(packed).to(_dev())
    out8, grad = plan.loss_backward(x)
    for b, phi in enumerate(phis):
        N = len(phi)
        M = 1 << int(np.ceil(np.log2(2 * N)))
        o8u, gu = g.af_loss_backward(torch.from_numpy(phi).to(_dev()), M, g.Window.full(N, M), loss)
        torch.cuda.synchronize()
        gb = grad[int(plan.offsets[b]):int(plan.offsets[b + 1])]
        assert torch.allclose(out8[b], o8u[0], rtol=2e-6, atol=0)
        assert float(torch.linalg.vector_norm(gb - gu[0]) / torch.linalg.vector_norm(gu[0])) <= 1e-5
    import tempfile, os
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    plan.autotune(x, cache_path=cache)
    assert os.path.exists(cache) and len(open(cache).read().split()) == 2 * len(plan.info())
    out8b, gradb = plan.loss_backward(x)
    torch.cuda.synchronize()
    assert torch.allclose(out8b, out8, rtol=2e-6, atol=0)
    assert float(torch.linalg.vector_norm(gradb - grad) / torch.linalg.vector_norm(grad)) <= 1e-5


def test_uneven_batch_1000_codes_128_to_8192():
    """1000 random-phase codes with lengths log-uniform in [128, 8192],
    M = next power of two >= 2N, PSL + ISL over all cells minus the zero-delay
    mainlobe, forward and backward in one plan.  Every code: finite scalars,
    E = N, sum_p dL/dphi_p = 0; the shortest codes fully against the oracle."""
    Ns = inputs.uneven_lengths(inputs.SEED_BASE + 4, 1000)
    phis, packed = _packed_phases(inputs.SEED_BASE + 4, Ns)
    loss = g.Loss(1.0, 1.0, 50.0, 1e-12)
    plan = g.BatchPlan(Ns, losses=[loss])
    info = plan.info()
    assert sorted(b["M"] for b in info) == sorted({1 << int(np.ceil(np.log2(2 * int(n)))) for n in Ns})
    x = torch.from_numpy(packed).to(_dev())
    out8, grad = plan.loss_backward(x)
    torch.cuda.synchronize()
    o8 = out8.cpu().numpy()
    gr = grad.cpu().numpy()
    assert np.all(np.isfinite(o8)) and np.all(np.isfinite(gr))
    assert np.all(np.abs(o8[:, 4] - Ns) <= 1e-6 * Ns * 10)
    for b in range(1000):
        gb = gr[plan.offsets[b]:plan.offsets[b + 1]]
        assert abs(gb.sum()) <= 1e-4 * np.linalg.norm(gb) * np.sqrt(len(gb))
    short = np.argsort(Ns)[:3]
    for b in short:
        N = int(Ns[b])
        M = 1 << int(np.ceil(np.log2(2 * N)))
        s = orc.signal_from_phase(phis[b].astype(np.float64))
        _, gp, ref8 = orc.grad(s, M, orc.full_window(N, M), 1.0, 1.0, 50.0, 1e-12)
        assert abs(o8[b, 0] - ref8[0]) <= L_TOL * abs(ref8[0])
        gb = gr[plan.offsets[b]:plan.offsets[b + 1]]
        assert np.linalg.norm(gb - gp) / np.linalg.norm(gp) <= G_TOL


@pytest.mark.slow
def test_uneven_batch_1000_codes_each_bucket_against_oracle():
    """The 1000-code plan of the workload above: in every M bucket (256 ...
    16384) the shortest code's loss scalars (1e-5) and gradient (1e-4
    relative L2) against the FP64 oracle.  The oracle's cost is dominated by
    the M = 16384 bucket's shortest code (N = 4122, about 5.6e11 complex
    multiply-adds: about 3 minutes on 16 threads)."""
    Ns = inputs.uneven_lengths(inputs.SEED_BASE + 4, 1000)
    phis, packed = _packed_phases(inputs.SEED_BASE + 4, Ns)
    loss = g.Loss(1.0, 1.0, 50.0, 1e-12)
    plan = g.BatchPlan(Ns, losses=[loss])
    out8, grad = plan.loss_backward(torch.from_numpy(packed).to(_dev()))
    torch.cuda.synchronize()
    o8, gr = out8.cpu().numpy(), grad.cpu().numpy()
    Ms = np.array([1 << int(np.ceil(np.log2(2 * int(n)))) for n in Ns])
    checked = []
    for M in sorted(set(Ms.tolist())):
        ids = np.nonzero(Ms == M)[0]
        b = int(ids[np.argmin(Ns[ids])])
        N = int(Ns[b])
        s = orc.signal_from_phase(phis[b].astype(np.float64))
        _, gp, ref8 = orc.grad(s, M, orc.full_window(N, M), 1.0, 1.0, 50.0, 1e-12)
        for i in (0, 1, 2, 3):
            assert abs(o8[b, i] - ref8[i]) <= L_TOL * abs(ref8[i]), (M, N, i, o8[b], ref8)
        assert o8[b, 5] == np.float32(ref8[5])
        gb = gr[plan.offsets[b]:plan.offsets[b + 1]]
        assert np.linalg.norm(gb - gp) / np.linalg.norm(gp) <= G_TOL, (M, N)
        checked.append(M)
    assert checked == [256, 512, 1024, 2048, 4096, 8192, 16384]


def _packed_complex(seed, Ns):
    zs = [inputs.random_complex(seed + i, 1, int(n))[0] for i, n in enumerate(Ns)]
    return zs, np.concatenate(zs)


def test_ragged_complex_batch_matches_oracle():
    """Complex signals of uneven length (Sec. 4.3's s in C^{B x N}, ragged):
    loss scalars and dL/dRe s + j dL/dIm s per waveform against the oracle,
    with default windows (two-pass: the row-0 box), masked windows, ISL-only
    losses (fused) and several M buckets."""
    Ns = [20, 33, 64, 100, 129, 200, 255, 47]
    Ms = [64, 128, 128, 256, 512, 512, 512, 128]
    windows = [g.Window.full(20, 64), g.Window.masked(10, 20), g.Window(-50, 63, -64, 63, 0, 0),
               g.Window(-30, 12, -128, 100, 0, 0), g.Window.full(129, 512), g.Window(5, 199, -256, 255, -1, -1),
               g.Window.full(255, 512), g.Window.masked(30, 40)]
    losses = [g.Loss(1.0, 1.0, 50.0, 1e-12), g.Loss(0.0, 1.0, 50.0, 1e-12), g.Loss(1.0, 0.5, 30.0, 1e-12),
              g.Loss(0.5, 2.0, 20.0, 1e-12), g.Loss(0.0, 1.0, 50.0, 1e-12), g.Loss(1.0, 1.0, 10.0, 1e-12),
              g.Loss(2.0, 1.0, 80.0, 1e-12), g.Loss(1.0, 1.0, 50.0, 1e-12)]
    zs, packed = _packed_complex(140, Ns)
    plan = g.BatchPlan(Ns, M=Ms, windows=windows, losses=losses, kind=g.GRAF_IN_COMPLEX)
    x = torch.from_numpy(packed).to(_dev())
    out8, grad = plan.loss_backward(x)
    only8 = plan.loss(x)
    torch.cuda.synchronize()
    out8, only8, grad = out8.cpu().numpy(), only8.cpu().numpy(), grad.cpu().numpy()
    for b, z in enumerate(zs):
        w, l = windows[b], losses[b]
        gs, _, o8 = orc.grad(z.astype(np.complex128), Ms[b], w.as_tuple(), l.w_psl, l.w_isl, l.beta, l.eps)
        for i in (0, 1, 2, 3):
            assert abs(out8[b, i] - o8[i]) <= L_TOL * max(abs(o8[i]), 1e-6), (b, i, out8[b], o8)
            assert abs(only8[b, i] - o8[i]) <= L_TOL * max(abs(o8[i]), 1e-6), (b, i, only8[b], o8)
        assert out8[b, 5] == np.float32(o8[5])
        gb = grad[plan.offsets[b]:plan.offsets[b + 1]]
        assert np.linalg.norm(gb - gs) / np.linalg.norm(gs) <= G_TOL, b
    dL = torch.linspace(-1.0, 2.0, len(Ns), device=_dev())
    _, g2 = plan.loss_backward(x, dL=dL)
    torch.cuda.synchronize()
    g2 = g2.cpu().numpy()
    for b in range(len(Ns)):
        sl = slice(int(plan.offsets[b]), int(plan.offsets[b + 1]))
        np.testing.assert_allclose(g2[sl], grad[sl] * float(dL[b]), rtol=1e-5, atol=1e-7)


@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_ragged_batch_forward_and_loss_only(kind):
    """graf_batch_forward: every waveform's Ahat window, packed, against the
    oracle; graf_batch_loss: the scalars of graf_batch_loss_backward."""
    Ns = [64, 100, 300, 31, 129]
    Ms = [128, 256, 1024, 64, 256]
    windows = [g.Window.full(64, 128), g.Window(-40, 20, -100, 27, 0, 1), g.Window(3, 150, -512, 511, 0, 0),
               g.Window.full(31, 64), g.Window(-128, -1, -5, 5, 0, 0)]
    if kind == "phase":
        sig, packed = _packed_phases(160, Ns)
        sigs = [orc.signal_from_phase(p.astype(np.float64)) for p in sig]
        gk = g.GRAF_IN_PHASE
    else:
        sig, packed = _packed_complex(160, Ns)
        sigs = [z.astype(np.complex128) for z in sig]
        gk = g.GRAF_IN_COMPLEX
    loss = g.Loss(1.0, 1.0, 50.0, 1e-12)
    plan = g.BatchPlan(Ns, M=Ms, windows=windows, losses=[loss], kind=gk)
    x = torch.from_numpy(packed).to(_dev())
    A, off = plan.forward(x)
    o8l = plan.loss(x)
    o8g, _ = plan.loss_backward(x)
    torch.cuda.synchronize()
    A = A.cpu().numpy()
    assert torch.allclose(o8l, o8g, rtol=2e-6, atol=0)
    for b, w in enumerate(windows):
        rows, cols = w.k_hi - w.k_lo + 1, w.m_hi - w.m_lo + 1
        assert off[b + 1] - off[b] == rows * cols
        want = orc.af_ahat(sigs[b], Ms[b], w.k_lo, w.k_hi, w.m_lo, w.m_hi, loss.eps)
        got = A[off[b]:off[b + 1]].reshape(rows, cols)
        assert np.abs(got - want).max() <= 1e-5, b
