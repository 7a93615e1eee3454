"""Pins for the oracle's optimiser: Adam against its textbook special cases
and against torch.optim.Adam (a library routine) in float64.  CPU only."""
import numpy as np
import pytest

import oracle as orc


def test_adam_constant_gradient_moves_by_lr():
    """With a constant gradient the bias-corrected moments are exact
    (m_hat = g, v_hat = g^2), so every step moves x by lr g / (|g| + eps)."""
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    x, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        x_prev = x
        x, m, v = orc.adam_update(x, m, v, g, t, lr=0.01)
        np.testing.assert_allclose(x_prev - x, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_matches_torch_adam():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x0 = rng.standard_normal(17)
    p = torch.tensor(x0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    x, m, v = x0.copy(), np.zeros(17), np.zeros(17)
    for t in range(1, 12):
        gr = rng.standard_normal(17) * (1 + t)
        opt.zero_grad()
        p.grad = torch.tensor(gr, dtype=torch.float64)
        opt.step()
        x, m, v = orc.adam_update(x, m, v, gr, t)
        np.testing.assert_allclose(x, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_oracle_optimiser_lowers_masked_isl():
    """A few Adam steps on the masked ISL of a random code lower it (the
    gradient points uphill and Adam steps against it)."""
    from paper_2506_22935_gb300 import inputs
    N, M = 32, 64
    phi0 = inputs.random_phases(5, 1, N)[0].astype(np.float64)
    win = (-8, 8, -8, 8, 0, 0)
    _, hist = orc.optimize_phases(phi0, M, win, 0.0, 1.0, 50.0, 1e-12, steps=15, lr=0.02)
    assert hist[-1] < hist[0]
