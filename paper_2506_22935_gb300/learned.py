"""Learned proposal of initial phase codes (the paper's Sec. 6.1 pipeline: a
network maps design parameters to a waveform, the GRAF layer scores it).

``ProposalMLP`` is an MLP spec[8] -> 512 -> 512 -> 1024 phases whose forward,
backward and optimiser run in the library's kernels (BF16 tensor-core GEMMs,
FP32 accumulation and master weights, Adam from ``graf_adam_step``).  Design
specs (delay and Doppler mask half-widths, PSL/ISL weights, noise) come from
``inputs.design_specs``; training labels are codes optimised on the GPU by
``PhaseOptimizer`` over each spec's own mask and loss (a ragged batch plan);
``time_to_target`` compares how many optimiser steps the proposal and a random
initialisation need to reach a masked-ISL target.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import graf as g
from . import inputs
from .optim import Adam, PhaseOptimizer

N_CODE, M_CODE = 1024, 2048


class ProposalMLP:
    def __init__(self, seed: int = 0, device=None, lr: float = 1e-3):
        g.load()
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        n = g.graf_mlp_param_count()
        self.master = torch.from_numpy(inputs.mlp_init_params(seed).astype(np.float32)).to(self.device)
        assert self.master.numel() == n
        self.bf16 = torch.empty(n, dtype=torch.bfloat16, device=self.device)
        self.grad = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.m = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.state = torch.zeros(g.graf_adam_state_bytes(), dtype=torch.uint8, device=self.device)
        self.hp = Adam(lr=lr).c()
        self._acts = None
        self._rows = 0
        self._cast()

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _cast(self):
        st = g.graf_mlp_cast_params(self.master.data_ptr(), self.bf16.data_ptr(), self._stream())
        if st != 0:
            raise g.GrafError(st, "graf_mlp_cast_params")

    def _activations(self, rows):
        if self._acts is None or self._rows < rows:
            self._acts = torch.empty(g.graf_mlp_activation_bytes(rows), dtype=torch.uint8, device=self.device)
            self._rows = rows
        return self._acts

    def forward(self, feats: torch.Tensor) -> torch.Tensor:
        """phases [rows, 1024] for spec features [rows, 8] (float32, CUDA)."""
        feats = feats.contiguous()
        rows = feats.shape[0]
        out = torch.empty((rows, g.GRAF_MLP_OUT), dtype=torch.float32, device=self.device)
        st = g.graf_mlp_forward(feats.data_ptr(), rows, self.master.data_ptr(), self.bf16.data_ptr(),
                                out.data_ptr(), self._activations(rows).data_ptr(), self._stream())
        if st != 0:
            raise g.GrafError(st, "graf_mlp_forward")
        return out

    def train_step(self, feats: torch.Tensor, targets: torch.Tensor, loss_out: torch.Tensor | None = None):
        """One Adam step on the mean phase label loss of a minibatch."""
        rows = feats.shape[0]
        phases = self.forward(feats)
        st = g.graf_mlp_label_loss(phases.data_ptr(), targets.contiguous().data_ptr(), rows, 1.0 / rows,
                                   None if loss_out is None else loss_out.data_ptr(), self._acts.data_ptr(),
                                   self._stream())
        if st != 0:
            raise g.GrafError(st, "graf_mlp_label_loss")
        st = g.graf_mlp_backward(rows, self.master.data_ptr(), self.bf16.data_ptr(), self._acts.data_ptr(),
                                 self.grad.data_ptr(), self._stream())
        if st != 0:
            raise g.GrafError(st, "graf_mlp_backward")
        st = g.graf_adam_step(self.master.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr(),
                              self.master.numel(), self.hp, self.step.data_ptr(), self.state.data_ptr(),
                              self._stream())
        if st != 0:
            raise g.GrafError(st, "graf_adam_step")
        self._cast()
        return phases

    def train_graf_step(self, feats: torch.Tensor, plan: "g.BatchPlan", ws: torch.Tensor, out8: torch.Tensor,
                        dphi: torch.Tensor):
        """One Adam step of the Sec. 6.1 pipeline: spec -> MLP -> phases ->
        GRAF loss of each spec's own window and weights (``plan``, one
        waveform of length 1024 per spec row) -> dL/dphi -> MLP backward.
        ``out8`` [rows, 8] receives the per-spec loss records."""
        rows = feats.shape[0]
        stream = self._stream()
        phases = self.forward(feats)
        st = g.graf_batch_loss_backward(plan.handle, phases.data_ptr(), out8.data_ptr(), None, dphi.data_ptr(),
                                        ws.data_ptr(), ws.numel(), stream)
        if st != 0:
            raise g.GrafError(st, "graf_batch_loss_backward")
        st = g.graf_mlp_set_output_grad(dphi.data_ptr(), rows, self._acts.data_ptr(), stream)
        if st != 0:
            raise g.GrafError(st, "graf_mlp_set_output_grad")
        st = g.graf_mlp_backward(rows, self.master.data_ptr(), self.bf16.data_ptr(), self._acts.data_ptr(),
                                 self.grad.data_ptr(), stream)
        if st != 0:
            raise g.GrafError(st, "graf_mlp_backward")
        st = g.graf_adam_step(self.master.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr(),
                              self.master.numel(), self.hp, self.step.data_ptr(), self.state.data_ptr(), stream)
        if st != 0:
            raise g.GrafError(st, "graf_adam_step")
        self._cast()
        return phases


class GrafTrainer:
    """End-to-end training of a ProposalMLP through the GRAF layer on a fixed
    set of training specs, split once into groups of ``group`` specs, each
    with its own batch plan (window and loss per spec); an epoch visits the
    groups in a fresh random order.  One workspace serves every plan."""

    def __init__(self, mlp: ProposalMLP, specs, group: int = 256, isl_only: bool = True, seed: int = 0):
        self.mlp, self.group = mlp, group
        dev = mlp.device
        count = len(specs["K"])
        self.feats = torch.from_numpy(inputs.spec_features(specs)).to(dev)
        self.plans = []
        nb = 256
        for c0 in range(0, count - group + 1, group):
            sub = {k: v[c0:c0 + group] for k, v in specs.items()}
            windows, losses = spec_windows_losses(sub, isl_only)
            plan = g.BatchPlan([N_CODE] * group, M=[M_CODE] * group, windows=windows, losses=losses, device=dev)
            nb = max(nb, g.graf_batch_workspace_bytes(plan.handle))
            self.plans.append((c0, plan))
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.out8 = torch.empty((group, 8), dtype=torch.float32, device=dev)
        self.dphi = torch.empty((group, N_CODE), dtype=torch.float32, device=dev)
        self.rng = np.random.default_rng(seed)

    def epoch(self) -> float:
        """One pass over the groups; returns the mean loss of the last group."""
        for i in self.rng.permutation(len(self.plans)):
            c0, plan = self.plans[i]
            self.mlp.train_graf_step(self.feats[c0:c0 + self.group], plan, self.ws, self.out8, self.dphi)
        return float(self.out8[:, 0].mean())

    def close(self):
        for _, plan in self.plans:
            plan.close()
        self.plans = []


def spec_windows_losses(specs, isl_only=False, beta=50.0):
    windows, losses = [], []
    for i in range(len(specs["K"])):
        windows.append(g.Window.masked(int(specs["K"][i]), int(specs["Mw"][i])))
        w_psl = 0.0 if isl_only else float(specs["w_psl"][i])
        w_isl = 1.0 if isl_only else float(specs["w_isl"][i])
        losses.append(g.Loss(w_psl, w_isl, beta, 1e-12))
    return windows, losses


def lfm_init(count: int) -> np.ndarray:
    """A deterministic starting code for the label optimiser: the discrete
    chirp pi n^2 / N for every spec."""
    return np.tile(inputs.lfm_phases(N_CODE), (count, 1))


def common_init(count: int, seed: int) -> np.ndarray:
    """The label optimiser's starting code: one seeded random phase code,
    the same for every spec, so that each spec's label is that code carried
    to its own optimum and labels vary with the spec rather than with the
    start (a learnable map)."""
    return np.tile(inputs.random_phases(seed, 1, N_CODE)[0], (count, 1))


def optimise_codes(specs, phi0: np.ndarray, steps: int, isl_only=False, device=None, graph=True, chunk=1024,
                   step_events=False):
    """Adam (lr 1e-2) on each spec's own masked loss from phi0 [count, N].
    Returns (codes [count, N], loss history [steps, count]) as numpy; with
    step_events (count <= chunk), also the GPU time in ms from the start of
    the run to the end of each step, [steps], from a CUDA event recorded after
    every step (the steps are then enqueued one by one)."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    count = phi0.shape[0]
    if step_events and count > chunk:
        raise ValueError("per-step events need the specs in one chunk")
    codes = np.empty_like(phi0, dtype=np.float32)
    hist = np.empty((steps, count), dtype=np.float32)
    step_ms = None
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        sub = {k: v[c0:c1] for k, v in specs.items()}
        windows, losses = spec_windows_losses(sub, isl_only)
        plan = g.BatchPlan([N_CODE] * (c1 - c0), M=[M_CODE] * (c1 - c0), windows=windows, losses=losses,
                           device=device)
        phi = torch.from_numpy(np.ascontiguousarray(phi0[c0:c1], dtype=np.float32)).to(device)
        opt = PhaseOptimizer(phi.view(-1), plan=plan, history_len=steps)
        if step_events:
            stream = torch.cuda.current_stream(device)
            start = torch.cuda.Event(enable_timing=True)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
            torch.cuda.synchronize(device)
            start.record(stream)
            for i in range(steps):
                opt.enqueue_step()
                evs[i].record(stream)
            torch.cuda.synchronize(device)
            step_ms = np.array([start.elapsed_time(e) for e in evs])
        else:
            opt.run(steps, graph=graph)
        torch.cuda.synchronize(device)
        codes[c0:c1] = phi.cpu().numpy()
        hist[:, c0:c1] = opt.history.cpu().numpy()
        plan.close()
    if step_events:
        return codes, hist, step_ms
    return codes, hist


def steps_to_target(hist: np.ndarray, target: np.ndarray) -> np.ndarray:
    """First step index (1-based, steps taken) whose loss is <= target, per
    column; hist.shape[0] + 1 where it never gets there."""
    ok = hist <= target[None, :]
    first = np.where(ok.any(axis=0), ok.argmax(axis=0), hist.shape[0])
    return first + 1


def masked_isl_targets(specs, steps=500, seeds=4, seed_base=7000, device=None) -> np.ndarray:
    """Per spec, the target T: the median over `seeds` random initialisations
    of the masked ISL after `steps` Adam steps of the plain optimiser."""
    finals = []
    for s in range(seeds):
        phi0 = inputs.random_phases(seed_base + s, len(specs["K"]), N_CODE)
        _, h = optimise_codes(specs, phi0, steps, isl_only=True, device=device)
        finals.append(h[-1])
    return np.median(np.stack(finals), axis=0)


def random_run(specs, steps=500, seed=7004, device=None):
    """The plain optimiser from one more random initialisation, timed per
    step: (loss history [steps, count], ms to the end of each step)."""
    phi_r = inputs.random_phases(seed, len(specs["K"]), N_CODE)
    _, h, ms = optimise_codes(specs, phi_r, steps, isl_only=True, device=device, step_events=True)
    return h, ms


def _run_time(ms, s):
    """GPU time to the end of the step whose loss first meets the target
    (s, 1-based); the whole run plus one step where it never does."""
    return np.where(s <= len(ms), ms[np.minimum(s, len(ms)) - 1], ms[-1] * (1.0 + 1.0 / len(ms)))


def time_to_target(mlp: ProposalMLP, specs, target: np.ndarray, random: tuple, steps=500, device=None):
    """Per held-out spec: the GPU time the optimiser needs to bring the spec
    to its target T (masked_isl_targets) from the MLP proposal -- the
    batch's MLP inference, timed with CUDA events, plus the run -- and from a
    random initialisation (random_run).  Both runs take every spec in one
    batch with a CUDA event after each step: a spec's time is the batch's
    measured time to the end of the step whose loss evaluation first meets T;
    a spec that does not reach T within `steps` is charged the whole run plus
    one step.  Returns numpy arrays and timings."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    feats = torch.from_numpy(inputs.spec_features(specs)).to(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mlp.forward(feats)  # warm-up
    torch.cuda.synchronize(device)
    e0.record()
    prop = mlp.forward(feats)
    e1.record()
    torch.cuda.synchronize(device)
    mlp_ms = e0.elapsed_time(e1)
    prop = np.mod(prop.cpu().numpy(), 2 * math.pi).astype(np.float32)
    _, h_learned, ms_l = optimise_codes(specs, prop, steps, isl_only=True, device=device, step_events=True)
    h_random, ms_r = random
    s_l = steps_to_target(h_learned, target)
    s_r = steps_to_target(h_random, target)
    return dict(target=target, steps_learned=s_l, steps_random=s_r, isl0_learned=h_learned[0],
                isl0_random=h_random[0], final_learned=h_learned[-1], final_random=h_random[-1],
                time_learned_ms=mlp_ms + _run_time(ms_l, s_l), time_random_ms=_run_time(ms_r, s_r),
                mlp_ms=mlp_ms, run_ms_learned=float(ms_l[-1]), run_ms_random=float(ms_r[-1]), steps=steps)
