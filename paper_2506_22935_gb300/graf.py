"""Python binding of ``libgraf.so`` (the C ABI in ``include/graf.h``).

Two layers:

* ``graf_*`` functions with the C names and arguments: pure ctypes marshalling
  of raw device pointers (ints), sizes and structs; they return the status
  code.  Every step of the computation runs in the library's CUDA kernels.
* torch conveniences (``af_forward``, ``af_loss``, ``af_backward``,
  ``af_loss_backward``, ``GrafAFLoss``): allocate outputs and workspaces with
  torch, pass torch's current stream, and raise on a non-zero status.  Torch
  is used for device memory and streams only.

There is no CPU fallback: if the library is missing or cannot be loaded, the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgraf.so")

GRAF_OK = 0
GRAF_ERR_DEVICE_FLAG = 6
GRAF_IN_COMPLEX = 0
GRAF_IN_PHASE = 1
GRAF_LOSS_OUT = 8
GRAF_M_MIN = 8
GRAF_M_MAX = 16384
GRAF_MLP_IN = 8
GRAF_MLP_OUT = 1024


class GrafError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {graf_status_string(status)} (status {status})")


class graf_window_t(ctypes.Structure):
    _fields_ = [("k_lo", ctypes.c_int32), ("k_hi", ctypes.c_int32), ("m_lo", ctypes.c_int32),
                ("m_hi", ctypes.c_int32), ("k_ml", ctypes.c_int32), ("m_ml", ctypes.c_int32)]


class graf_loss_t(ctypes.Structure):
    _fields_ = [("w_psl", ctypes.c_float), ("w_isl", ctypes.c_float), ("beta", ctypes.c_float),
                ("eps", ctypes.c_float)]


class graf_adam_t(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_sz = ctypes.c_size_t

# C signatures: name -> (restype, argtypes)
_SIGS = {
    "graf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "graf_version": (_i32, []),
    "graf_get_device_error_word": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), _vp]),
    "graf_get_device_error": (ctypes.c_int, [_vp]),
    "graf_af_forward": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, ctypes.c_float,
                                       _vp, _vp]),
    "graf_af_loss_workspace_bytes": (_sz, [_i32, _i32, _i32, graf_window_t]),
    "graf_af_loss": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, graf_loss_t, _vp,
                                    _vp, _sz, _vp]),
    "graf_af_backward_workspace_bytes": (_sz, [_i32, _i32, _i32, graf_window_t]),
    "graf_af_backward": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, graf_loss_t,
                                        _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_af_loss_backward": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t,
                                             graf_loss_t, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_af_loss_backward_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t,
                                                     graf_loss_t, _vp, _vp, _vp, _vp, _vp]),
    "graf_paf_forward": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, _i32, _vp, _vp]),
    "graf_paf_workspace_bytes": (_sz, [_i32, _i32, graf_window_t]),
    "graf_paf_loss": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, graf_loss_t, _vp, _vp,
                                     _sz, _vp]),
    "graf_paf_loss_backward": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, graf_loss_t,
                                              _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_spectral_variance": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, ctypes.c_float, _vp, _vp, _vp, _vp,
                                              _i32, _vp]),
    "graf_composite_terms": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, ctypes.c_float, ctypes.c_float,
                                            ctypes.c_float, ctypes.c_float, _vp, _vp, _vp, _vp, _i32, _vp]),
    "graf_af_match_workspace_bytes": (_sz, [_i32, _i32, _i32, graf_window_t]),
    "graf_af_match": (ctypes.c_int, [_vp, ctypes.c_int, _i32, _i32, _i32, graf_window_t, _vp, ctypes.c_float,
                                     ctypes.c_float, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp]),
    "graf_batch_plan_create": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _i32, ctypes.c_int, _vp]),
    "graf_batch_plan_create_scenarios": (ctypes.c_int, [_i32, _vp, _i32, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "graf_batch_plan_destroy": (ctypes.c_int, [_vp]),
    "graf_batch_workspace_bytes": (_sz, [_vp]),
    "graf_batch_plan_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _i32]),
    "graf_batch_loss_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_batch_loss_backward_complex": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_batch_loss": (ctypes.c_int, [_vp, _vp, _vp, _vp, _sz, _vp]),
    "graf_batch_af_offsets": (ctypes.c_int, [_vp, _vp]),
    "graf_batch_forward": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "graf_batch_autotune": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _sz, _vp, ctypes.c_char_p]),
    "graf_mlp_param_count": (_sz, []),
    "graf_mlp_activation_bytes": (_sz, [_i32]),
    "graf_mlp_cast_params": (ctypes.c_int, [_vp, _vp, _vp]),
    "graf_mlp_forward": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "graf_mlp_label_loss": (ctypes.c_int, [_vp, _vp, _i32, ctypes.c_float, _vp, _vp, _vp]),
    "graf_mlp_set_output_grad": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "graf_mlp_backward": (ctypes.c_int, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "graf_adam_state_bytes": (_sz, []),
    "graf_adam_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int64, graf_adam_t, _vp, _vp, _vp]),
    "graf_record_loss": (ctypes.c_int, [_vp, _i32, _vp, _i32, _vp, _vp]),
}

EXPORTED = tuple(_SIGS)


def load(path: str | None = None):
    """Load libgraf.so (built by ``__graft_entry__.build()``).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"libgraf.so not found at {p}: run __graft_entry__.build() first "
                                  "(the CUDA library is required; there is no fallback)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


# ---------------------------------------------------------------- raw ABI
def graf_status_string(status: int) -> str:
    return load().graf_status_string(int(status)).decode()


def graf_version() -> int:
    return load().graf_version()


GRAF_DEVERR_ENERGY = 1
GRAF_DEVERR_NONFINITE = 2


def graf_get_device_error(stream) -> int:
    return load().graf_get_device_error(stream)


def device_error_word(device=None) -> int:
    """Takes (reads and clears) the device error word after the work queued
    on the current stream: GRAF_DEVERR_* bits, 0 if nothing was raised."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    w = ctypes.c_uint32(0)
    _check(load().graf_get_device_error_word(ctypes.byref(w), _stream(dev)), "graf_get_device_error_word")
    return int(w.value)


def graf_af_forward(x, kind, B, N, M, w, eps, af_out, stream) -> int:
    return load().graf_af_forward(x, kind, B, N, M, w, eps, af_out, stream)


def graf_spectral_variance(x, kind, B, N, weight, out8, sv_out, grad_s, grad_phi, accumulate, stream) -> int:
    return load().graf_spectral_variance(x, kind, B, N, weight, out8, sv_out, grad_s, grad_phi, accumulate,
                                         stream)


def spectral_variance(x, weight: float = 1.0):
    """(SV [B], weighted gradient) of the normalised power spectrum (Eq. 25)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    sv = torch.empty(B, dtype=torch.float32, device=x.device)
    grad = torch.empty((B, N), dtype=torch.float32 if kind == GRAF_IN_PHASE else torch.complex64, device=x.device)
    gs = grad.data_ptr() if kind == GRAF_IN_COMPLEX else None
    gp = grad.data_ptr() if kind == GRAF_IN_PHASE else None
    _check(graf_spectral_variance(x.data_ptr(), kind, B, N, float(weight), None, sv.data_ptr(), gs, gp, 0,
                                  _stream(x.device)), "graf_spectral_variance")
    return sv, grad


def graf_composite_terms(x, kind, B, N, gamma, eps, w_width, w_const, out8, terms_out, grad_s, grad_phi,
                         accumulate, stream) -> int:
    return load().graf_composite_terms(x, kind, B, N, gamma, eps, w_width, w_const, out8, terms_out, grad_s,
                                       grad_phi, accumulate, stream)


def composite_terms(x, gamma: float = 50.0, eps: float = 0.0, w_width: float = 1.0, w_const: float = 0.0):
    """({W, V} [B, 2], gradient of w_width W + w_const V): the differentiable
    mainlobe width (Sec. 5.1) and var(|s|) (Eq. 22)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    terms = torch.empty((B, 2), dtype=torch.float32, device=x.device)
    grad = torch.empty((B, N), dtype=torch.float32 if kind == GRAF_IN_PHASE else torch.complex64, device=x.device)
    gs = grad.data_ptr() if kind == GRAF_IN_COMPLEX else None
    gp = grad.data_ptr() if kind == GRAF_IN_PHASE else None
    _check(graf_composite_terms(x.data_ptr(), kind, B, N, float(gamma), float(eps), float(w_width), float(w_const),
                                None, terms.data_ptr(), gs, gp, 0, _stream(x.device)), "graf_composite_terms")
    return terms, grad


def graf_af_match_workspace_bytes(B, N, M, w) -> int:
    return load().graf_af_match_workspace_bytes(B, N, M, w)


def graf_af_match(x, kind, B, N, M, w, target, weight, eps, loss_out, out8, grad_s, grad_phi, accumulate,
                  workspace, workspace_bytes, stream) -> int:
    return load().graf_af_match(x, kind, B, N, M, w, target, weight, eps, loss_out, out8, grad_s, grad_phi,
                                accumulate, workspace, workspace_bytes, stream)


def af_match(x, M: int, window: Window, target, weight: float = 1.0, eps: float = 1e-12):
    """(sum (Ahat^2 - target)^2 [B], gradient of weight * that sum)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    nb = graf_af_match_workspace_bytes(B, N, M, window.c())
    if nb == 0:
        raise GrafError(1, "graf_af_match_workspace_bytes")
    ws = _workspace(nb, x.device)
    target = target.contiguous().to(torch.float32)
    loss = torch.empty(B, dtype=torch.float32, device=x.device)
    grad = torch.empty((B, N), dtype=torch.float32 if kind == GRAF_IN_PHASE else torch.complex64, device=x.device)
    gs = grad.data_ptr() if kind == GRAF_IN_COMPLEX else None
    gp = grad.data_ptr() if kind == GRAF_IN_PHASE else None
    _check(graf_af_match(x.data_ptr(), kind, B, N, M, window.c(), target.data_ptr(), float(weight), float(eps),
                         loss.data_ptr(), None, gs, gp, 0, ws.data_ptr(), ws.numel(), _stream(x.device)),
           "graf_af_match")
    return loss, grad


def graf_paf_forward(x, kind, B, N, sign, normalise, chi_out, stream) -> int:
    return load().graf_paf_forward(x, kind, B, N, sign, normalise, chi_out, stream)


def graf_paf_workspace_bytes(B, N, w) -> int:
    return load().graf_paf_workspace_bytes(B, N, w)


def graf_paf_loss(x, kind, B, N, sign, w, l, out8, workspace, workspace_bytes, stream) -> int:
    return load().graf_paf_loss(x, kind, B, N, sign, w, l, out8, workspace, workspace_bytes, stream)


def graf_paf_loss_backward(x, kind, B, N, sign, w, l, out8, dL, grad_s, grad_phi, workspace, workspace_bytes,
                           stream) -> int:
    return load().graf_paf_loss_backward(x, kind, B, N, sign, w, l, out8, dL, grad_s, grad_phi, workspace,
                                         workspace_bytes, stream)


def graf_af_loss_workspace_bytes(B, N, M, w) -> int:
    return load().graf_af_loss_workspace_bytes(B, N, M, w)


def graf_af_loss(x, kind, B, N, M, w, l, out8, workspace, workspace_bytes, stream) -> int:
    return load().graf_af_loss(x, kind, B, N, M, w, l, out8, workspace, workspace_bytes, stream)


def graf_af_backward_workspace_bytes(B, N, M, w) -> int:
    return load().graf_af_backward_workspace_bytes(B, N, M, w)


def graf_af_backward(x, kind, B, N, M, w, l, saved8, dL, grad_s, grad_phi, workspace, workspace_bytes,
                     stream) -> int:
    return load().graf_af_backward(x, kind, B, N, M, w, l, saved8, dL, grad_s, grad_phi, workspace,
                                   workspace_bytes, stream)


def graf_af_loss_backward(x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, workspace, workspace_bytes,
                          stream) -> int:
    return load().graf_af_loss_backward(x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, workspace,
                                        workspace_bytes, stream)


def graf_af_loss_backward_noalloc(x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, stream) -> int:
    """graf_af_loss_backward on the library's fixed scratch array (no workspace
    argument, nothing allocated): for callers that cannot allocate device
    memory.  Calls that may overlap on the GPU must be serialised."""
    return load().graf_af_loss_backward_noalloc(x, kind, B, N, M, w, l, out8, dL, grad_s, grad_phi, stream)


def graf_batch_plan_create(B, N_host, M_host, w_host, l_host, losses_per_waveform, kind, plan_out) -> int:
    return load().graf_batch_plan_create(B, N_host, M_host, w_host, l_host, losses_per_waveform, kind, plan_out)


def graf_batch_plan_destroy(plan) -> int:
    return load().graf_batch_plan_destroy(plan)


def graf_batch_workspace_bytes(plan) -> int:
    return load().graf_batch_workspace_bytes(plan)


def graf_batch_plan_info(plan, n_buckets, M_out, rpt_out, items_out, fused_out, capacity) -> int:
    return load().graf_batch_plan_info(plan, n_buckets, M_out, rpt_out, items_out, fused_out, capacity)


def graf_batch_plan_create_scenarios(S, src, B_src, N_src, M, w, l, kind, plan) -> int:
    return load().graf_batch_plan_create_scenarios(S, src, B_src, N_src, M, w, l, kind, plan)


def graf_batch_loss_backward(plan, phi, out8, dL, grad_phi, workspace, workspace_bytes, stream) -> int:
    return load().graf_batch_loss_backward(plan, phi, out8, dL, grad_phi, workspace, workspace_bytes, stream)


def graf_batch_loss_backward_complex(plan, s, out8, dL, grad_s, workspace, workspace_bytes, stream) -> int:
    return load().graf_batch_loss_backward_complex(plan, s, out8, dL, grad_s, workspace, workspace_bytes, stream)


def graf_batch_loss(plan, x, out8, workspace, workspace_bytes, stream) -> int:
    return load().graf_batch_loss(plan, x, out8, workspace, workspace_bytes, stream)


def graf_batch_af_offsets(plan, af_off_host) -> int:
    return load().graf_batch_af_offsets(plan, af_off_host)


def graf_batch_forward(plan, x, af_out, stream) -> int:
    return load().graf_batch_forward(plan, x, af_out, stream)


def graf_batch_autotune(plan, phi, out8, grad_phi, workspace, workspace_bytes, stream, cache_path) -> int:
    return load().graf_batch_autotune(plan, phi, out8, grad_phi, workspace, workspace_bytes, stream, cache_path)


def graf_mlp_param_count() -> int:
    return load().graf_mlp_param_count()


def graf_mlp_activation_bytes(rows) -> int:
    return load().graf_mlp_activation_bytes(rows)


def graf_mlp_cast_params(master, params_bf16, stream) -> int:
    return load().graf_mlp_cast_params(master, params_bf16, stream)


def graf_mlp_forward(spec, rows, master, params_bf16, phases, activations, stream) -> int:
    return load().graf_mlp_forward(spec, rows, master, params_bf16, phases, activations, stream)


def graf_mlp_label_loss(phases, target, rows, scale, loss, activations, stream) -> int:
    return load().graf_mlp_label_loss(phases, target, rows, scale, loss, activations, stream)


def graf_mlp_set_output_grad(dphases, rows, activations, stream) -> int:
    return load().graf_mlp_set_output_grad(dphases, rows, activations, stream)


def graf_mlp_backward(rows, master, params_bf16, activations, grad, stream) -> int:
    return load().graf_mlp_backward(rows, master, params_bf16, activations, grad, stream)


def graf_adam_state_bytes() -> int:
    return load().graf_adam_state_bytes()


def graf_adam_step(x, m, v, grad, count, hp, step, state, stream) -> int:
    return load().graf_adam_step(x, m, v, grad, count, hp, step, state, stream)


def graf_record_loss(out8, B, history, history_len, step, stream) -> int:
    return load().graf_record_loss(out8, B, history, history_len, step, stream)


# ---------------------------------------------------------------- helpers
@dataclass(frozen=True)
class Window:
    """Delay/Doppler window and mainlobe box (see ``graf_window_t``)."""
    k_lo: int
    k_hi: int
    m_lo: int
    m_hi: int
    k_ml: int = 0
    m_ml: int = 0

    @staticmethod
    def full(N: int, M: int, k_ml: int = 0, m_ml: int | None = None) -> "Window":
        """Every delay and Doppler bin.  Default mainlobe box: k = 0 and
        |m| < M/N, the zero-delay Doppler mainlobe of a unit-modulus code."""
        if m_ml is None:
            m_ml = max(M // N - 1, 0)
        return Window(-(N - 1), N - 1, -(M // 2), M // 2 - 1, k_ml, m_ml)

    @staticmethod
    def periodic(N: int, k_ml: int = 0, m_ml: int = 0) -> "Window":
        """Every delay and Doppler bin of the periodic AF (both in [-N/2,
        N/2-1]) minus the box (default: the origin)."""
        return Window(-(N // 2), N // 2 - 1, -(N // 2), N // 2 - 1, k_ml, m_ml)

    @staticmethod
    def masked(K: int, Mw: int, k_ml: int = 0, m_ml: int = 0) -> "Window":
        """|k| <= K, |m| <= Mw, minus the box (default: the origin only)."""
        return Window(-K, K, -Mw, Mw, k_ml, m_ml)

    def c(self) -> graf_window_t:
        return graf_window_t(self.k_lo, self.k_hi, self.m_lo, self.m_hi, self.k_ml, self.m_ml)

    def as_tuple(self):
        return (self.k_lo, self.k_hi, self.m_lo, self.m_hi, self.k_ml, self.m_ml)


@dataclass(frozen=True)
class Loss:
    """L = w_psl PSL_soft + w_isl ISL with soft-max temperature beta; with
    beta = math.inf, L = w_psl PSL_hard + w_isl ISL (the hard maximum of
    Eq. 18, differentiated through its arg-max cell)."""
    w_psl: float = 1.0
    w_isl: float = 1.0
    beta: float = 50.0
    eps: float = 1e-12

    @staticmethod
    def hard(w_psl: float = 1.0, w_isl: float = 0.0, eps: float = 1e-12) -> "Loss":
        return Loss(w_psl, w_isl, float("inf"), eps)

    def c(self) -> graf_loss_t:
        return graf_loss_t(self.w_psl, self.w_isl, self.beta, self.eps)


def _torch():
    import torch
    return torch


def _prep(x):
    """-> (tensor, kind, B, N) for complex64 signals or float32 phases, [B,N] or [N]."""
    torch = _torch()
    if not x.is_cuda:
        raise ValueError("graf: input must be a CUDA tensor")
    if x.dim() == 1:
        x = x.unsqueeze(0)
    if x.dim() != 2:
        raise ValueError("graf: input must be [B, N] or [N]")
    if x.dtype == torch.complex64:
        kind = GRAF_IN_COMPLEX
    elif x.dtype == torch.float32:
        kind = GRAF_IN_PHASE
    else:
        raise ValueError("graf: input must be complex64 (signal) or float32 (phases)")
    x = x.contiguous()
    return x, kind, x.shape[0], x.shape[1]


def _stream(device):
    return _torch().cuda.current_stream(device).cuda_stream


def _check(st, what):
    if st != GRAF_OK:
        raise GrafError(st, what)


def _workspace(nbytes, device):
    torch = _torch()
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def af_forward(x, M: int, window: Window | None = None, eps: float = 1e-12):
    """Ahat over the window, float32 [B, k_hi-k_lo+1, m_hi-m_lo+1]."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    w = window or Window.full(N, M)
    out = torch.empty((B, w.k_hi - w.k_lo + 1, w.m_hi - w.m_lo + 1), dtype=torch.float32, device=x.device)
    _check(graf_af_forward(x.data_ptr(), kind, B, N, M, w.c(), eps, out.data_ptr(), _stream(x.device)),
           "graf_af_forward")
    return out


def af_loss(x, M: int, window: Window | None = None, loss: Loss = Loss(), workspace=None):
    """Loss scalars [B, 8] = (L, PSL_soft, ISL, PSL_hard, E, |Omega|, S_p, 0)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    w = window or Window.full(N, M)
    nb = graf_af_loss_workspace_bytes(B, N, M, w.c())
    if nb == 0:
        raise GrafError(1, "graf_af_loss_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= nb else _workspace(nb, x.device)
    out = torch.empty((B, GRAF_LOSS_OUT), dtype=torch.float32, device=x.device)
    _check(graf_af_loss(x.data_ptr(), kind, B, N, M, w.c(), loss.c(), out.data_ptr(), ws.data_ptr(),
                        ws.numel(), _stream(x.device)), "graf_af_loss")
    return out


def af_backward(x, M: int, window: Window | None, loss: Loss, saved8, dL=None, want: str = "auto",
                workspace=None):
    """Gradient w.r.t. the input.  want='phi' (phase input) -> float32 [B,N];
    want='s' -> complex64 [B,N] (dL/dRe s + j dL/dIm s); 'auto' picks by dtype."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    w = window or Window.full(N, M)
    if want == "auto":
        want = "phi" if kind == GRAF_IN_PHASE else "s"
    nb = graf_af_backward_workspace_bytes(B, N, M, w.c())
    if nb == 0:
        raise GrafError(1, "graf_af_backward_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= nb else _workspace(nb, x.device)
    saved8 = saved8.contiguous()
    dl = None if dL is None else dL.reshape(B).to(torch.float32).contiguous()
    gs = torch.empty((B, N), dtype=torch.complex64, device=x.device) if want == "s" else None
    gp = torch.empty((B, N), dtype=torch.float32, device=x.device) if want == "phi" else None
    _check(graf_af_backward(x.data_ptr(), kind, B, N, M, w.c(), loss.c(), saved8.data_ptr(),
                            None if dl is None else dl.data_ptr(), None if gs is None else gs.data_ptr(),
                            None if gp is None else gp.data_ptr(), ws.data_ptr(), ws.numel(),
                            _stream(x.device)), "graf_af_backward")
    return gp if want == "phi" else gs


def af_loss_backward(x, M: int, window: Window | None = None, loss: Loss = Loss(), dL=None,
                     workspace=None, out8=None, grad=None):
    """One forward+backward step; returns (out8 [B,8], grad)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    w = window or Window.full(N, M)
    nb = graf_af_backward_workspace_bytes(B, N, M, w.c())
    if nb == 0:
        raise GrafError(1, "graf_af_backward_workspace_bytes")
    ws = workspace if workspace is not None and workspace.numel() >= nb else _workspace(nb, x.device)
    out8 = out8 if out8 is not None else torch.empty((B, GRAF_LOSS_OUT), dtype=torch.float32, device=x.device)
    if grad is None:
        grad = torch.empty((B, N), dtype=torch.float32 if kind == GRAF_IN_PHASE else torch.complex64,
                           device=x.device)
    dl = None if dL is None else dL.reshape(B).to(torch.float32).contiguous()
    gs = grad.data_ptr() if kind == GRAF_IN_COMPLEX else None
    gp = grad.data_ptr() if kind == GRAF_IN_PHASE else None
    _check(graf_af_loss_backward(x.data_ptr(), kind, B, N, M, w.c(), loss.c(), out8.data_ptr(),
                                 None if dl is None else dl.data_ptr(), gs, gp, ws.data_ptr(), ws.numel(),
                                 _stream(x.device)), "graf_af_loss_backward")
    return out8, grad


def paf_forward(x, sign: int = 1, normalise: bool = True):
    """Periodic AF chi [B, N, N] (Eq. 7, Algorithm 1), fftshift order, over
    max chi = E^2 if normalise."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    out = torch.empty((B, N, N), dtype=torch.float32, device=x.device)
    _check(graf_paf_forward(x.data_ptr(), kind, B, N, int(sign), 1 if normalise else 0, out.data_ptr(),
                            _stream(x.device)), "graf_paf_forward")
    return out


def paf_loss_backward(x, window: Window | None = None, loss: Loss = Loss(), sign: int = 1, dL=None):
    """Loss scalars and gradient of the periodic AF (default window: every
    delay and Doppler bin minus the origin); returns (out8 [B,8], grad)."""
    torch = _torch()
    x, kind, B, N = _prep(x)
    w = window or Window.periodic(N)
    nb = graf_paf_workspace_bytes(B, N, w.c())
    if nb == 0:
        raise GrafError(1, "graf_paf_workspace_bytes")
    ws = _workspace(nb, x.device)
    out8 = torch.empty((B, GRAF_LOSS_OUT), dtype=torch.float32, device=x.device)
    grad = torch.empty((B, N), dtype=torch.float32 if kind == GRAF_IN_PHASE else torch.complex64, device=x.device)
    dl = None if dL is None else dL.reshape(B).to(torch.float32).contiguous()
    gs = grad.data_ptr() if kind == GRAF_IN_COMPLEX else None
    gp = grad.data_ptr() if kind == GRAF_IN_PHASE else None
    _check(graf_paf_loss_backward(x.data_ptr(), kind, B, N, int(sign), w.c(), loss.c(), out8.data_ptr(),
                                  None if dl is None else dl.data_ptr(), gs, gp, ws.data_ptr(), ws.numel(),
                                  _stream(x.device)), "graf_paf_loss_backward")
    return out8, grad


class BatchPlan:
    """A ragged batch plan (graf_batch_plan_create) with torch-allocated
    workspace: waveform b has length N[b], Doppler length M[b] (default the
    next power of two >= 2 N[b]), window windows[b] (default: all bins minus
    the zero-delay mainlobe) and loss losses[b] (or one loss for all)."""

    def __init__(self, N, M=None, windows=None, losses=None, device=None, kind: int = GRAF_IN_PHASE):
        torch = _torch()
        import numpy as np
        self.kind = kind
        self.N = np.asarray(N, dtype=np.int32)
        self.B = len(self.N)
        Nc = np.ascontiguousarray(self.N)
        Mc = None if M is None else np.ascontiguousarray(np.asarray(M, dtype=np.int32))
        wc = None
        if windows is not None:
            wc = (graf_window_t * self.B)(*[w.c() for w in windows])
        if losses is None:
            losses = [Loss()]
        per = 1 if len(losses) == self.B and self.B > 1 else 0
        lc = (graf_loss_t * len(losses))(*[l.c() for l in losses])
        h = ctypes.c_void_p()
        st = graf_batch_plan_create(self.B, Nc.ctypes.data, None if Mc is None else Mc.ctypes.data,
                                    None if wc is None else ctypes.addressof(wc), ctypes.addressof(lc), per,
                                    kind, ctypes.byref(h))
        _check(st, "graf_batch_plan_create")
        self.handle = h
        self.offsets = np.concatenate([[0], np.cumsum(self.N.astype(np.int64))])
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self._ws = None

    @classmethod
    def scenarios(cls, N_src, src, windows, losses, M=None, device=None, kind: int = GRAF_IN_PHASE) -> "BatchPlan":
        """A multi-scenario plan (Eq. 24): entry b scores source src[b] of
        lengths N_src with windows[b] and losses[b]; loss_backward then takes
        the packed sources, the per-entry weights lambda as dL, and returns
        the per-source summed gradient."""
        torch = _torch()
        import numpy as np
        self = cls.__new__(cls)
        self.kind = kind
        src = np.ascontiguousarray(np.asarray(src, dtype=np.int32))
        Ns = np.ascontiguousarray(np.asarray(N_src, dtype=np.int32))
        S = len(src)
        self.B = S
        self.N = Ns[src]
        Mc = None if M is None else np.ascontiguousarray(np.asarray(M, dtype=np.int32))
        wc = (graf_window_t * S)(*[w.c() for w in windows])
        lc = (graf_loss_t * S)(*[l.c() for l in losses])
        h = ctypes.c_void_p()
        _check(graf_batch_plan_create_scenarios(S, src.ctypes.data, len(Ns), Ns.ctypes.data,
                                                None if Mc is None else Mc.ctypes.data, ctypes.addressof(wc),
                                                ctypes.addressof(lc), kind, ctypes.byref(h)),
               "graf_batch_plan_create_scenarios")
        self.handle = h
        self.offsets = np.concatenate([[0], np.cumsum(Ns.astype(np.int64))])  # of the sources
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self._ws = None
        return self

    def workspace(self):
        torch = _torch()
        nb = graf_batch_workspace_bytes(self.handle)
        if self._ws is None or self._ws.numel() < nb:
            self._ws = torch.empty(max(nb, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def info(self):
        n = ctypes.c_int32()
        cap = 32
        arrs = [(ctypes.c_int32 * cap)() for _ in range(4)]
        _check(graf_batch_plan_info(self.handle, ctypes.byref(n), *[ctypes.addressof(a) for a in arrs], cap),
               "graf_batch_plan_info")
        return [dict(M=arrs[0][i], rows_per_tile=arrs[1][i], items=arrs[2][i], fused=bool(arrs[3][i]))
                for i in range(n.value)]

    def loss_backward(self, x_packed, dL=None, out8=None, grad=None):
        """(out8 [B, 8], gradient packed like the input): dL/dphi for a phase
        plan (float32 input), dL/dRe s + j dL/dIm s for a complex plan
        (complex64 input)."""
        torch = _torch()
        out8 = out8 if out8 is not None else torch.empty((self.B, 8), dtype=torch.float32, device=self.device)
        grad = grad if grad is not None else torch.empty_like(x_packed)
        ws = self.workspace()
        fn = graf_batch_loss_backward if self.kind == GRAF_IN_PHASE else graf_batch_loss_backward_complex
        st = fn(self.handle, x_packed.data_ptr(), out8.data_ptr(), None if dL is None else dL.data_ptr(),
                grad.data_ptr(), ws.data_ptr(), ws.numel(), torch.cuda.current_stream(self.device).cuda_stream)
        _check(st, fn.__name__)
        return out8, grad

    def loss(self, x_packed, out8=None):
        """Loss scalars [B, 8] alone (graf_batch_loss)."""
        torch = _torch()
        out8 = out8 if out8 is not None else torch.empty((self.B, 8), dtype=torch.float32, device=self.device)
        ws = self.workspace()
        _check(graf_batch_loss(self.handle, x_packed.data_ptr(), out8.data_ptr(), ws.data_ptr(), ws.numel(),
                               torch.cuda.current_stream(self.device).cuda_stream), "graf_batch_loss")
        return out8

    def af_offsets(self):
        import numpy as np
        off = np.zeros(self.B + 1, dtype=np.int64)
        _check(graf_batch_af_offsets(self.handle, off.ctypes.data), "graf_batch_af_offsets")
        return off

    def forward(self, x_packed):
        """Every waveform's Ahat window, packed (split with af_offsets())."""
        torch = _torch()
        off = self.af_offsets()
        out = torch.empty(int(off[-1]), dtype=torch.float32, device=self.device)
        _check(graf_batch_forward(self.handle, x_packed.data_ptr(), out.data_ptr(),
                                  torch.cuda.current_stream(self.device).cuda_stream), "graf_batch_forward")
        return out, off

    def autotune(self, phi_packed, cache_path=None):
        torch = _torch()
        out8 = torch.empty((self.B, 8), dtype=torch.float32, device=self.device)
        grad = torch.empty_like(phi_packed)
        # room for the smallest tiles tried
        ws = torch.empty(max(4 * graf_batch_workspace_bytes(self.handle), 1 << 20), dtype=torch.uint8,
                         device=self.device)
        st = graf_batch_autotune(self.handle, phi_packed.data_ptr(), out8.data_ptr(), grad.data_ptr(),
                                 ws.data_ptr(), ws.numel(), torch.cuda.current_stream(self.device).cuda_stream,
                                 None if cache_path is None else str(cache_path).encode())
        _check(st, "graf_batch_autotune")
        self._ws = None

    def close(self):
        if getattr(self, "handle", None):
            graf_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    torch = _torch()

    class GrafAFLoss(torch.autograd.Function):
        """L(x) per waveform (float32 [B]) with the library's Wirtinger backward.

        x: float32 phases [B, N] or complex64 signals [B, N].  The gradient
        follows PyTorch's complex convention (dL/dRe + j dL/dIm)."""

        @staticmethod
        def forward(ctx, x, M, window, loss):
            out8 = af_loss(x, M, window, loss)
            ctx.save_for_backward(x, out8)
            ctx.cfg = (M, window, loss)
            ctx.mark_non_differentiable(out8)
            return out8[:, 0].clone(), out8

        @staticmethod
        def backward(ctx, g_l, g_out8):
            x, out8 = ctx.saved_tensors
            M, window, loss = ctx.cfg
            if g_l is None:
                return None, None, None, None
            g = af_backward(x, M, window, loss, out8, dL=g_l)
            return g.reshape(x.shape), None, None, None

    return GrafAFLoss


_autograd_cls = None


def GrafAFLoss():
    """The torch.autograd.Function class (created lazily so importing this
    module does not import torch)."""
    global _autograd_cls
    if _autograd_cls is None:
        _autograd_cls = _make_autograd()
    return _autograd_cls


def af_loss_autograd(x, M: int, window: Window | None = None, loss: Loss = Loss()):
    """Differentiable per-waveform loss [B] (and the detached scalars [B, 8])."""
    xx = x if x.dim() == 2 else x.unsqueeze(0)
    w = window or Window.full(xx.shape[1], M)
    return GrafAFLoss().apply(xx, M, w, loss)
