"""Multi-scenario loss (Eq. 24) through a scenario batch plan: one launch
scores each source waveform under several windows and loss weights, and the
gradient per source is the lambda-weighted sum, against the FP64 oracle."""
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


def test_scenario_plan_matches_weighted_oracle_sum():
    N_src = [100, 60, 33]
    src = [0, 0, 1, 0, 1, 2, 2]
    lam = np.array([0.5, 1.0, 2.0, 0.3, 1.5, 0.7, 1.1], dtype=np.float32)
    M_of = lambda N: 1 << int(np.ceil(np.log2(2 * N)))
    windows, losses, Ms = [], [], []
    for b, j in enumerate(src):
        N, M = N_src[j], M_of(N_src[j])
        Ms.append(M)
        if b % 3 == 0:      # the whole AF minus the zero-delay mainlobe
            windows.append(g.Window.full(N, M))
            losses.append(g.Loss(1.0, 1.0, 50.0, 1e-12))
        elif b % 3 == 1:    # a range-Doppler box around a target, ISL only
            windows.append(g.Window(-(N // 4), N // 4, -(M // 8), M // 8, 0, 0))
            losses.append(g.Loss(0.0, 1.0, 50.0, 1e-12))
        else:               # a velocity band, PSL + ISL
            windows.append(g.Window(-(N - 1), N - 1, M // 16, M // 4, -1, -1))
            losses.append(g.Loss(0.5, 1.0, 30.0, 1e-12))
    phis = [inputs.random_phases(101 + j, 1, N)[0] for j, N in enumerate(N_src)]
    x = torch.from_numpy(np.concatenate(phis)).to("cuda:0")
    plan = g.BatchPlan.scenarios(N_src, src, windows, losses, M=Ms)
    dL = torch.from_numpy(lam).to("cuda:0")
    out8, grad = plan.loss_backward(x, dL=dL)
    torch.cuda.synchronize()
    out8, grad = out8.cpu().numpy(), grad.cpu().numpy()
    plan.close()
    ref = [np.zeros(N) for N in N_src]
    for b, j in enumerate(src):
        lo = losses[b]
        s = np.exp(1j * phis[j].astype(np.float64))
        _, gp, o = oracle.grad(s, Ms[b], windows[b].as_tuple(), lo.w_psl, lo.w_isl, lo.beta, lo.eps)
        assert abs(out8[b, 0] - o[0]) <= 1e-5 * abs(o[0]), (b, out8[b, 0], o[0])
        ref[j] += lam[b] * gp
    off = np.concatenate([[0], np.cumsum(N_src)])
    for j in range(len(N_src)):
        gj = grad[off[j]:off[j + 1]]
        assert np.linalg.norm(gj - ref[j]) <= 1e-4 * np.linalg.norm(ref[j]), j
