"""Learned proposal MLP: forward, label loss and backward against the FP64
reference (with the same BF16 roundings), and a short end-to-end training
run on GPU-optimised labels."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2506_22935_gb300 import _build, inputs
from paper_2506_22935_gb300 import graf as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    g.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_mlp_forward_loss_backward_match_reference():
    from paper_2506_22935_gb300.learned import ProposalMLP
    dev = torch.device("cuda:0")
    rows = 37  # not a multiple of the 64-row tile: ragged tail
    net = ProposalMLP(seed=3)
    rng = np.random.default_rng(5)
    flat = inputs.mlp_init_params(3) + 0.02 * rng.standard_normal(omlp.param_count())
    flat[:16 * 512].reshape(16, 512)[8:, :] = 0.0
    net.master.copy_(torch.from_numpy(flat.astype(np.float32)))
    net._cast()
    feats = inputs.spec_features(inputs.design_specs(11, rows))
    target = inputs.random_phases(12, rows, 1024)
    out = net.forward(torch.from_numpy(feats).to(dev))
    loss = torch.empty(rows, device=dev)
    st = g.graf_mlp_label_loss(out.data_ptr(), torch.from_numpy(target).to(dev).data_ptr(), rows, 1.0 / rows,
                               loss.data_ptr(), net._acts.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 0
    assert g.graf_mlp_backward(rows, net.master.data_ptr(), net.bf16.data_ptr(), net._acts.data_ptr(),
                               net.grad.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    flat32 = flat.astype(np.float32).astype(np.float64)
    ref, cache = omlp.forward(feats.astype(np.float64), flat32)
    assert _rel(out.cpu().numpy(), ref) <= 2e-3
    rl, rg = omlp.label_loss(out.cpu().numpy().astype(np.float64), target.astype(np.float64), 1.0 / rows)
    np.testing.assert_allclose(loss.cpu().numpy(), rl, rtol=1e-4, atol=1e-5)
    gref = omlp.backward(cache, rg)
    assert _rel(net.grad.cpu().numpy(), gref) <= 1e-2


def test_short_training_lowers_label_loss():
    from paper_2506_22935_gb300.learned import ProposalMLP, lfm_init, optimise_codes
    dev = torch.device("cuda:0")
    specs = inputs.design_specs(21, 256)
    codes, hist = optimise_codes(specs, lfm_init(256), steps=100, device=dev)
    assert np.all(hist[-1] < hist[0])
    net = ProposalMLP(seed=1, lr=1e-3)
    feats = torch.from_numpy(inputs.spec_features(specs)).to(dev)
    tgt = torch.from_numpy(codes).to(dev)
    loss = torch.empty(256, device=dev)
    first = None
    for it in range(150):
        net.train_step(feats, tgt, loss_out=loss)
        if it == 0:
            first = float(loss.mean())
    last = float(loss.mean())
    assert last < 0.8 * first, (first, last)
