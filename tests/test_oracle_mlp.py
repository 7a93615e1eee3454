"""Pins for the MLP reference and its label loss: torch autograd (a library
routine) for the backward, finite differences and invariances for the loss,
torch's bfloat16 cast for the rounding.  CPU only."""
import numpy as np
import pytest

from oracle import mlp
from paper_2506_22935_gb300 import inputs

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    x = np.concatenate([inputs.normal(3, 5000) * 10.0 ** np.arange(-4, 6).repeat(500),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)


def test_backward_matches_torch_autograd():
    rng = np.random.default_rng(0)
    flat = inputs.mlp_init_params(7) + 0.01 * rng.standard_normal(mlp.param_count())
    spec = rng.standard_normal((5, mlp.IN))
    dout = rng.standard_normal((5, mlp.OUT))
    out, cache = mlp.forward(spec, flat, bf16_round=False)
    got = mlp.backward(cache, dout)
    pt = torch.tensor(flat, dtype=torch.float64, requires_grad=True)
    P = {}
    o = 0
    for name, shape in mlp.SHAPES:
        n = int(np.prod(shape))
        P[name] = pt[o:o + n].reshape(shape)
        o += n
    x = torch.zeros((5, mlp.IN_PAD), dtype=torch.float64)
    x[:, :mlp.IN] = torch.tensor(spec)
    gelu = torch.nn.functional.gelu
    y = gelu(gelu(x @ P["W1"] + P["b1"]) @ P["W2"] + P["b2"]) @ P["W3"] + P["b3"]
    np.testing.assert_allclose(out, y.detach().numpy(), rtol=1e-12, atol=1e-12)
    (y * torch.tensor(dout)).sum().backward()
    np.testing.assert_allclose(got, pt.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_label_loss_invariances_and_gradient():
    rng = np.random.default_rng(1)
    n = 64
    t = rng.uniform(0, 2 * np.pi, (3, n))
    p = t + 0.3 * rng.standard_normal((3, n))
    l0, g0 = mlp.label_loss(p, t)
    l1, _ = mlp.label_loss(p + 1.234, t)          # global phase
    l2, _ = mlp.label_loss(-p, t)                 # conjugate proposal
    np.testing.assert_allclose(l1, l0, rtol=1e-12)
    np.testing.assert_allclose(l2, l0, rtol=1e-12)
    assert np.all(mlp.label_loss(t, t)[0] < 1e-12)
    h = 1e-6
    fd = np.zeros_like(p)
    for b in range(3):
        for i in range(n):
            e = np.zeros_like(p)
            e[b, i] = h
            fd[b, i] = (mlp.label_loss(p + e, t)[0][b] - mlp.label_loss(p - e, t)[0][b]) / (2 * h)
    np.testing.assert_allclose(g0, fd, rtol=1e-6, atol=1e-9)
