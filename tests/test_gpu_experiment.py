"""The paper's experiment loss (Sec. 7.1.1, Eq. 25) on the GPU optimiser:
periodic AF PSL + lambda alpha spectral variance, Adam lr 0.01, against the
FP64 restatement step by step."""
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


@pytest.mark.parametrize("lam", [0.0, 0.5, 2.0])
@pytest.mark.parametrize("graph", [False, True])
def test_experiment_steps_match_oracle(lam, graph):
    from paper_2506_22935_gb300.optim import Adam, PhaseOptimizer
    B, N, steps = 2, 64, 30
    lp = (1.0, 0.0, 100.0)
    win = g.Window.periodic(N)
    phi0 = inputs.random_phases(81, B, N)
    phi = torch.from_numpy(phi0.copy()).to("cuda:0")
    opt = PhaseOptimizer(phi, window=win, loss=g.Loss(*lp, 1e-12), adam=Adam(lr=1e-2), history_len=steps,
                         periodic_sign=1, spectral_weight=2000.0 * lam)
    opt.run(steps, graph=graph)
    torch.cuda.synchronize()
    hist = opt.history.cpu().numpy()
    got = phi.cpu().numpy()
    for b in range(B):
        ref_phi, ref_hist = oracle.optimize_experiment(phi0[b], win.as_tuple(), *lp, 1e-12, 2000.0 * lam, steps)
        np.testing.assert_allclose(hist[:, b], ref_hist, rtol=2e-4)
        assert np.abs(got[b] - ref_phi).max() <= 2e-4
    assert np.all(hist[-1] < hist[0])
