"""On-device phase-code optimisation: the gradient refinement of Sec. 6.2 (Eq. 23)
with Adam (Sec. 7.1.2), every step on the GPU through the C ABI.

One step = ``graf_af_loss_backward`` (fused loss + dL/dphi) ->
``graf_record_loss`` (loss curve kept on the device) -> ``graf_adam_step``
(update with the step count held on the device).  ``PhaseOptimizer.run``
captures a whole run of steps in one CUDA graph and replays it, so the host
enqueues nothing per step.  Torch provides the device memory and the stream.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import graf as g


@dataclass(frozen=True)
class Adam:
    lr: float = 1e-2
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def c(self) -> g.graf_adam_t:
        return g.graf_adam_t(self.lr, self.beta1, self.beta2, self.eps)


class PhaseOptimizer:
    """Adam on phases phi [B, N] (float32, CUDA, updated in place) for the loss
    ``loss`` over ``window`` with Doppler length M; or, with ``plan`` (a
    graf.BatchPlan), on the packed phases of a ragged batch whose windows and
    losses the plan holds (phi then [sum N] or [B, N] for equal lengths).

    ``periodic_sign`` (+1 or -1) selects the paper's periodic AF (Eq. 7, M = N)
    instead of the aperiodic one; ``spectral_weight`` adds lambda alpha times
    the spectral variance of Eq. 25 to the loss and its gradient (the
    experiment loss of Sec. 7.1.1)."""

    def __init__(self, phi: torch.Tensor, M: int = 0, window: g.Window | None = None, loss: g.Loss | None = None,
                 adam: Adam = Adam(), history_len: int = 1000, plan: "g.BatchPlan | None" = None,
                 periodic_sign: int | None = None, spectral_weight: float = 0.0):
        if phi.dtype != torch.float32 or not phi.is_cuda or not phi.is_contiguous():
            raise ValueError("phi must be a contiguous CUDA float32 tensor")
        g.load()
        self.phi, self.M, self.window, self.loss, self.adam, self.plan = phi, M, window, loss, adam, plan
        self.periodic_sign, self.spectral_weight = periodic_sign, float(spectral_weight)
        dev = phi.device
        if plan is None:
            if phi.dim() != 2:
                raise ValueError("phi must be [B, N]")
            self.B, self.N = phi.shape
            if periodic_sign is not None:
                self.M = self.N
                self.nb = g.graf_paf_workspace_bytes(self.B, self.N, window.c())
            else:
                self.nb = g.graf_af_backward_workspace_bytes(self.B, self.N, M, window.c())
            if self.nb == 0:
                raise g.GrafError(1, "graf_af_backward_workspace_bytes")
            self.ws = torch.empty(self.nb, dtype=torch.uint8, device=dev)
            self._wc, self._lc = window.c(), loss.c()
        else:
            self.B, self.N = plan.B, int(plan.offsets[-1])
            self.ws = plan.workspace()
            self.nb = self.ws.numel()
        self.m = torch.zeros_like(phi)
        self.v = torch.zeros_like(phi)
        self.grad = torch.zeros_like(phi)
        self.out8 = torch.zeros((self.B, 8), dtype=torch.float32, device=dev)
        self.step_counter = torch.zeros(1, dtype=torch.int32, device=dev)
        self.state = torch.zeros(g.graf_adam_state_bytes(), dtype=torch.uint8, device=dev)
        self.history = torch.full((history_len, self.B), float("nan"), dtype=torch.float32, device=dev)
        self._hp = adam.c()
        self._graphs = {}

    def enqueue_step(self) -> None:
        """Enqueue one optimisation step on torch's current stream."""
        st = torch.cuda.current_stream(self.phi.device).cuda_stream
        if self.plan is None and self.periodic_sign is not None:
            r = g.graf_paf_loss_backward(self.phi.data_ptr(), g.GRAF_IN_PHASE, self.B, self.N, self.periodic_sign,
                                         self._wc, self._lc, self.out8.data_ptr(), None, None, self.grad.data_ptr(),
                                         self.ws.data_ptr(), self.nb, st)
        elif self.plan is None:
            r = g.graf_af_loss_backward(self.phi.data_ptr(), g.GRAF_IN_PHASE, self.B, self.N, self.M, self._wc,
                                        self._lc, self.out8.data_ptr(), None, None, self.grad.data_ptr(),
                                        self.ws.data_ptr(), self.nb, st)
        else:
            r = g.graf_batch_loss_backward(self.plan.handle, self.phi.data_ptr(), self.out8.data_ptr(), None,
                                           self.grad.data_ptr(), self.ws.data_ptr(), self.nb, st)
        if r != 0:
            raise g.GrafError(r, "graf_af_loss_backward")
        if self.spectral_weight != 0.0:
            if self.plan is not None:
                raise ValueError("the spectral term needs equal-length waveforms")
            r = g.graf_spectral_variance(self.phi.data_ptr(), g.GRAF_IN_PHASE, self.B, self.N, self.spectral_weight,
                                         self.out8.data_ptr(), None, None, self.grad.data_ptr(), 1, st)
            if r != 0:
                raise g.GrafError(r, "graf_spectral_variance")
        r = g.graf_record_loss(self.out8.data_ptr(), self.B, self.history.data_ptr(), self.history.shape[0],
                               self.step_counter.data_ptr(), st)
        if r != 0:
            raise g.GrafError(r, "graf_record_loss")
        r = g.graf_adam_step(self.phi.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), self.grad.data_ptr(),
                             self.phi.numel(), self._hp, self.step_counter.data_ptr(), self.state.data_ptr(), st)
        if r != 0:
            raise g.GrafError(r, "graf_adam_step")

    def capture(self, steps: int) -> torch.cuda.CUDAGraph:
        """A CUDA graph of `steps` consecutive steps (captured once, cached)."""
        if steps not in self._graphs:
            side = torch.cuda.Stream(self.phi.device)
            side.wait_stream(torch.cuda.current_stream(self.phi.device))
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=side):
                for _ in range(steps):
                    self.enqueue_step()
            torch.cuda.current_stream(self.phi.device).wait_stream(side)
            self._graphs[steps] = graph
        return self._graphs[steps]

    def run(self, steps: int, graph: bool = True) -> None:
        """Run `steps` steps: one graph replay, or one enqueue per step."""
        if graph:
            self.capture(steps).replay()
        else:
            for _ in range(steps):
                self.enqueue_step()

    def reset(self, phi0: torch.Tensor) -> None:
        """Restart from phi0 with fresh moments and step count (graphs stay valid)."""
        self.phi.copy_(phi0)
        self.m.zero_()
        self.v.zero_()
        self.step_counter.zero_()
        self.history.fill_(float("nan"))
