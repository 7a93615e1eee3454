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


def test_graf_chain_gradient_matches_reference():
    """Spec -> MLP -> phases -> masked ISL (batch plan) -> dL/dphi -> MLP
    backward, against the FP64 AF adjoint chained into the FP64/BF16 MLP
    reference at the same phases."""
    import oracle
    from paper_2506_22935_gb300.learned import ProposalMLP, spec_windows_losses
    dev = torch.device("cuda:0")
    specs = inputs.design_specs(31, 3)
    specs["K"] = np.array([20, 33, 47], dtype=np.int32)
    specs["Mw"] = np.array([9, 16, 30], dtype=np.int32)
    windows, losses = spec_windows_losses(specs, isl_only=True)
    plan = g.BatchPlan([1024] * 3, M=[2048] * 3, windows=windows, losses=losses, device=dev)
    net = ProposalMLP(seed=4)
    feats = inputs.spec_features(specs)
    phases = net.forward(torch.from_numpy(feats).to(dev))
    out8, dphi = plan.loss_backward(phases.view(-1))
    stream = torch.cuda.current_stream().cuda_stream
    assert g.graf_mlp_set_output_grad(dphi.data_ptr(), 3, net._acts.data_ptr(), stream) == 0
    assert g.graf_mlp_backward(3, net.master.data_ptr(), net.bf16.data_ptr(), net._acts.data_ptr(),
                               net.grad.data_ptr(), stream) == 0
    torch.cuda.synchronize()
    plan.close()
    ph = phases.cpu().numpy().astype(np.float64)
    dref = np.empty_like(ph)
    for b in range(3):
        lo = losses[b]
        _, gp, o8 = oracle.grad(np.exp(1j * ph[b]), 2048, windows[b].as_tuple(), lo.w_psl, lo.w_isl, lo.beta,
                                lo.eps)
        dref[b] = gp
        np.testing.assert_allclose(out8[b, 0].item(), o8[0], rtol=1e-4)
    assert _rel(dphi.view(3, -1).cpu().numpy(), dref) <= 1e-4
    _, cache = omlp.forward(feats.astype(np.float64), net.master.cpu().numpy().astype(np.float64))
    assert _rel(net.grad.cpu().numpy(), omlp.backward(cache, dref)) <= 1e-2


def test_graf_training_lowers_masked_isl():
    from paper_2506_22935_gb300.learned import GrafTrainer, ProposalMLP
    specs = inputs.design_specs(41, 256)
    net = ProposalMLP(seed=2, lr=1e-3)
    tr = GrafTrainer(net, specs, group=256, isl_only=True)
    first = tr.epoch()
    for _ in range(60):
        last = tr.epoch()
    tr.close()
    assert last < 0.9 * first, (first, last)


def test_label_trained_proposal_reaches_the_target_sooner():
    """The learned pipeline at small scale, as the benchmark runs it: 256
    training specs labelled by the GPU optimiser (each spec's own loss, 500
    Adam steps from one common seeded code), the MLP trained on the (spec,
    label) pairs with the phase label loss, then 32 held-out specs: from the
    proposal the plain optimiser reaches the spec's masked-ISL target (the
    median of 4 random initialisations after 500 steps) in fewer steps, and
    less measured GPU time, than from a random initialisation, on the median
    held-out spec."""
    from paper_2506_22935_gb300 import learned
    dev = torch.device("cuda:0")
    train = inputs.design_specs(inputs.SEED_BASE + 40, 256)
    test = inputs.design_specs(inputs.SEED_BASE + 41, 32)
    codes, _ = learned.optimise_codes(train, learned.common_init(256, inputs.SEED_BASE + 42), 500, device=dev)
    net = learned.ProposalMLP(seed=5)
    feats = torch.from_numpy(inputs.spec_features(train)).to(dev)
    tgt = torch.from_numpy(codes).to(dev)
    for _ in range(300):
        net.train_step(feats, tgt)
    target = learned.masked_isl_targets(test, 500, device=dev)
    rand = learned.random_run(test, 500, device=dev)
    r = learned.time_to_target(net, test, target, rand, 500, device=dev)
    assert np.median(r["steps_learned"]) < np.median(r["steps_random"]), (r["steps_learned"], r["steps_random"])
    assert np.median(r["time_learned_ms"] / r["time_random_ms"]) < 1.0
