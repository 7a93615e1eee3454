"""FP64 CPU oracle for the differentiable ambiguity function (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It loads ``graf_oracle.c``
(plain C, direct double sums, no FFT) through ctypes, compiling it with gcc on
first use, and shares no code with the CUDA library.

Conventions (paper Sec. 4.1, Eqs. 8, 11, 12, 17-19, 22):
  * ``beta = inf`` selects the hard PSL of Eq. 18, max over Omega of Ahat^2
    (the beta -> infinity limit of the log-sum-exp PSL), whose subgradient
    goes through one arg-max cell: the first in row-major window order.
  * ``s`` is complex128 of length N; ``phi`` float64 phases, s = exp(j phi).
  * windows are ``(k_lo, k_hi, m_lo, m_hi, k_ml, m_ml)``: delay and Doppler
    ranges (inclusive, Doppler in fftshift order [-M/2, M/2-1]) and the
    mainlobe box |k|<=k_ml and |m|<=m_ml that the losses exclude.
  * loss scalars ``out8`` = (L, PSL_soft, ISL, PSL_hard, E, |Omega|,
    sum_Omega p*Ahat^2, 0).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graf_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liborc.so`` (gcc, -O2)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp,
                               "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_signal_from_phase.argtypes = [_dp, _i64, _dp]
            lib.orc_energy.argtypes = [_dp, _i64]
            lib.orc_energy.restype = ctypes.c_double
            lib.orc_af_complex.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, _i64, _dp, ctypes.c_int]
            lib.orc_af_ahat.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, _i64, ctypes.c_double,
                                        _dp, ctypes.c_int]
            lib.orc_af_cells.argtypes = [_dp, _i64, _i64, _i64, _ip, _ip, ctypes.c_double, _dp]
            lib.orc_loss.argtypes = [_dp, _i64, _i64, _ip, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _dp, ctypes.c_int]
            lib.orc_grad.argtypes = [_dp, _i64, _i64, _ip, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, ctypes.c_int]
            lib.orc_fd_grad_phi.argtypes = [_dp, _i64, _i64, _ip, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                                            ctypes.c_int]
            lib.orc_fd_grad_s.argtypes = [_dp, _i64, _i64, _ip, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp,
                                          ctypes.c_int]
            _c = ctypes.c_int
            _d = ctypes.c_double
            lib.orc_paf_complex.argtypes = [_dp, _i64, _c, _i64, _i64, _i64, _i64, _dp]
            lib.orc_ploss.argtypes = [_dp, _i64, _c, _ip, _d, _d, _d, _d, _dp]
            lib.orc_pgrad.argtypes = [_dp, _i64, _c, _ip, _d, _d, _d, _d, _dp, _dp, _dp]
            lib.orc_pfd_grad_phi.argtypes = [_dp, _i64, _c, _ip, _d, _d, _d, _d, _d, _dp]
            lib.orc_match.argtypes = [_dp, _i64, _i64, _ip, _dp, _d, _d, _dp, _dp, _dp, _c]
            lib.orc_peak_cell.argtypes = [_dp, _i64, _i64, _ip, _d, _ip, _c]
            lib.orc_cell_grad.argtypes = [_dp, _i64, _i64, _i64, _i64, _d, _dp, _dp]
            lib.orc_ppeak_cell.argtypes = [_dp, _i64, _c, _ip, _d, _ip]
            lib.orc_pcell_grad.argtypes = [_dp, _i64, _c, _i64, _i64, _d, _dp, _dp]
            for f in ("orc_af_complex", "orc_af_ahat", "orc_af_cells", "orc_loss", "orc_grad",
                      "orc_fd_grad_phi", "orc_fd_grad_s", "orc_paf_complex", "orc_ploss", "orc_pgrad",
                      "orc_pfd_grad_phi", "orc_match", "orc_peak_cell", "orc_cell_grad", "orc_ppeak_cell",
                      "orc_pcell_grad"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _threads(nthreads):
    return int(nthreads) if nthreads else (os.cpu_count() or 1)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _s_buf(s):
    s = np.ascontiguousarray(np.asarray(s, dtype=np.complex128))
    return s, s.view(np.float64)


def _check(st, what):
    if st != 0:
        raise ValueError(f"oracle {what} failed with status {st}")


def full_window(N: int, M: int, k_ml: int = 0, m_ml=None):
    """All 2N-1 delays and all M Doppler bins.  ``m_ml=None`` gives the default
    mainlobe box of the full-AF workloads: k=0, |m| < M/N (first null of the
    zero-delay row of a unit-modulus code).  A box size of -1 excludes nothing."""
    if m_ml is None:
        m_ml = max(M // N - 1, 0)
    return (-(N - 1), N - 1, -(M // 2), M - 1 - M // 2, k_ml, m_ml)


def signal_from_phase(phi) -> np.ndarray:
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    out = np.empty(phi.shape[0], dtype=np.complex128)
    _load().orc_signal_from_phase(_ptr(phi), phi.shape[0], _ptr(out.view(np.float64)))
    return out


def energy(s) -> float:
    s, sv = _s_buf(s)
    return float(_load().orc_energy(_ptr(sv), s.shape[0]))


def af_complex(s, M, k_lo, k_hi, m_lo, m_hi, nthreads=None) -> np.ndarray:
    """X[k,m] over the window, shape (k_hi-k_lo+1, m_hi-m_lo+1), complex128."""
    s, sv = _s_buf(s)
    X = np.empty((k_hi - k_lo + 1, m_hi - m_lo + 1), dtype=np.complex128)
    st = _load().orc_af_complex(_ptr(sv), s.shape[0], M, k_lo, k_hi, m_lo, m_hi,
                                _ptr(X.view(np.float64)), _threads(nthreads))
    _check(st, "af_complex")
    return X


def af_ahat(s, M, k_lo, k_hi, m_lo, m_hi, eps, nthreads=None) -> np.ndarray:
    """Energy-normalised, eps-stabilised |X| over the window (float64)."""
    s, sv = _s_buf(s)
    A = np.empty((k_hi - k_lo + 1, m_hi - m_lo + 1), dtype=np.float64)
    st = _load().orc_af_ahat(_ptr(sv), s.shape[0], M, k_lo, k_hi, m_lo, m_hi, float(eps),
                             _ptr(A), _threads(nthreads))
    _check(st, "af_ahat")
    return A


def af_cells(s, M, ks, ms, eps) -> np.ndarray:
    """Ahat at the listed (k, m) cells, each computed by its own direct sum."""
    s, sv = _s_buf(s)
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int64))
    ms = np.ascontiguousarray(np.asarray(ms, dtype=np.int64))
    out = np.empty(ks.shape[0], dtype=np.float64)
    st = _load().orc_af_cells(_ptr(sv), s.shape[0], M, ks.shape[0], ks.ctypes.data_as(_ip),
                              ms.ctypes.data_as(_ip), float(eps), _ptr(out))
    _check(st, "af_cells")
    return out


def _win(window):
    w = np.ascontiguousarray(np.asarray(window, dtype=np.int64))
    assert w.shape == (6,)
    return w


def loss(s, M, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, nthreads=None) -> np.ndarray:
    s, sv = _s_buf(s)
    w = _win(window)
    out = np.zeros(8, dtype=np.float64)
    st = _load().orc_loss(_ptr(sv), s.shape[0], M, w.ctypes.data_as(_ip), w_psl, w_isl, beta, eps,
                          _ptr(out), _threads(nthreads))
    _check(st, "loss")
    return out


def grad(s, M, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, nthreads=None):
    """Returns (grad_s complex128 = dL/dRe s + j dL/dIm s,
    grad_phi float64 = dL/dphi for s = exp(j phi), out8)."""
    s, sv = _s_buf(s)
    w = _win(window)
    N = s.shape[0]
    gs = np.zeros(N, dtype=np.complex128)
    gp = np.zeros(N, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    st = _load().orc_grad(_ptr(sv), N, M, w.ctypes.data_as(_ip), w_psl, w_isl, beta, eps,
                          _ptr(gs.view(np.float64)), _ptr(gp), _ptr(out), _threads(nthreads))
    _check(st, "grad")
    return gs, gp, out


def peak_cell(s, M, window, eps=1e-12, nthreads=None):
    """(k, m) of the arg-max of Ahat^2 over Omega that the hard PSL uses."""
    s, sv = _s_buf(s)
    w = _win(window)
    pk = np.zeros(2, dtype=np.int64)
    _check(_load().orc_peak_cell(_ptr(sv), s.shape[0], M, w.ctypes.data_as(_ip), eps, pk.ctypes.data_as(_ip),
                                 _threads(nthreads)), "peak_cell")
    return int(pk[0]), int(pk[1])


def cell_grad(s, M, k, m, eps=1e-12):
    """(grad_s, grad_phi) of one cell's Ahat^2[k, m] (conventions as grad)."""
    s, sv = _s_buf(s)
    N = s.shape[0]
    gs = np.zeros(N, dtype=np.complex128)
    gp = np.zeros(N, dtype=np.float64)
    _check(_load().orc_cell_grad(_ptr(sv), N, M, int(k), int(m), eps, _ptr(gs.view(np.float64)), _ptr(gp)),
           "cell_grad")
    return gs, gp


def fd_grad_phi(phi, M, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, h=1e-6,
                nthreads=None) -> np.ndarray:
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    w = _win(window)
    out = np.zeros(phi.shape[0], dtype=np.float64)
    st = _load().orc_fd_grad_phi(_ptr(phi), phi.shape[0], M, w.ctypes.data_as(_ip), w_psl, w_isl,
                                 beta, eps, h, _ptr(out), _threads(nthreads))
    _check(st, "fd_grad_phi")
    return out


def fd_grad_s(s, M, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, h=1e-6,
              nthreads=None) -> np.ndarray:
    s, sv = _s_buf(s)
    w = _win(window)
    out = np.zeros(s.shape[0], dtype=np.complex128)
    st = _load().orc_fd_grad_s(_ptr(sv), s.shape[0], M, w.ctypes.data_as(_ip), w_psl, w_isl, beta,
                               eps, h, _ptr(out.view(np.float64)), _threads(nthreads))
    _check(st, "fd_grad_s")
    return out


# ------------------------------------------------------------------ optimiser
def adam_update(x, m, v, g, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1), float64, returns (x, m, v):
    m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; x -= lr m_hat / (sqrt(v_hat) + eps),
    m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t).  t counts from 1."""
    x, m, v, g = (np.asarray(a, dtype=np.float64) for a in (x, m, v, g))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return x - lr * mh / (np.sqrt(vh) + eps), m, v


def optimize_phases(phi0, M, window, w_psl, w_isl, beta, eps, steps, lr=1e-2, beta1=0.9, beta2=0.999,
                    adam_eps=1e-8, nthreads=None):
    """Gradient refinement of the phases (the paper's Eq. 23 with Adam): per
    step the loss and dL/dphi of orc_grad, then one Adam update.  Returns
    (phi after `steps` steps, loss before each step)."""
    phi = np.asarray(phi0, dtype=np.float64).copy()
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    hist = []
    for t in range(1, steps + 1):
        _, gphi, out = grad(signal_from_phase(phi), M, window, w_psl, w_isl, beta, eps, nthreads)
        hist.append(out[0])
        phi, m, v = adam_update(phi, m, v, gphi, t, lr, beta1, beta2, adam_eps)
    return phi, np.array(hist)


# ----------------------------------------------------------- periodic AF
# The paper's own discrete AF (Sec. 3.1 Eq. 2, Sec. 4.1 Eq. 7, Algorithm 1):
# circular lag (n - k) mod N, N Doppler bins, exponent sign +1 (Eq. 7) or -1
# (the FFT of Algorithm 1); delays and Doppler bins in fftshift order
# [-N/2, N/2 - 1].

def full_pwindow(N: int, k_ml: int = 0, m_ml: int = 0):
    """Every delay and Doppler bin of the periodic AF; default box: the origin."""
    return (-(N // 2), N - 1 - N // 2, -(N // 2), N - 1 - N // 2, k_ml, m_ml)


def paf_complex(s, sign=1, k_lo=None, k_hi=None, m_lo=None, m_hi=None) -> np.ndarray:
    """X[k,m] over the window (default all), shape (rows, cols), complex128."""
    s, sv = _s_buf(s)
    N = s.shape[0]
    k_lo = -(N // 2) if k_lo is None else k_lo
    k_hi = N - 1 - N // 2 if k_hi is None else k_hi
    m_lo = -(N // 2) if m_lo is None else m_lo
    m_hi = N - 1 - N // 2 if m_hi is None else m_hi
    X = np.zeros((k_hi - k_lo + 1, m_hi - m_lo + 1), dtype=np.complex128)
    _check(_load().orc_paf_complex(_ptr(sv), N, int(sign), k_lo, k_hi, m_lo, m_hi, _ptr(X.view(np.float64))),
           "paf_complex")
    return X


def paf_chi(s, sign=1, normalise=True) -> np.ndarray:
    """chi = |X|^2 (Eq. 12), divided by E^2 = chi[0,0] = max chi if normalise
    (Eq. 17); [N][N], fftshift order (as in Algorithm 1)."""
    X = paf_complex(s, sign)
    chi = np.abs(X) ** 2
    if normalise:
        chi = chi / energy(s) ** 2
    return chi


def ploss(s, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, sign=1) -> np.ndarray:
    s, sv = _s_buf(s)
    w = _win(window)
    out = np.zeros(8, dtype=np.float64)
    _check(_load().orc_ploss(_ptr(sv), s.shape[0], int(sign), w.ctypes.data_as(_ip), w_psl, w_isl, beta, eps,
                             _ptr(out)), "ploss")
    return out


def pgrad(s, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, sign=1):
    """(grad_s, grad_phi, out8) of the periodic-AF loss, conventions as grad."""
    s, sv = _s_buf(s)
    w = _win(window)
    N = s.shape[0]
    gs = np.zeros(N, dtype=np.complex128)
    gp = np.zeros(N, dtype=np.float64)
    out = np.zeros(8, dtype=np.float64)
    _check(_load().orc_pgrad(_ptr(sv), N, int(sign), w.ctypes.data_as(_ip), w_psl, w_isl, beta, eps,
                             _ptr(gs.view(np.float64)), _ptr(gp), _ptr(out)), "pgrad")
    return gs, gp, out


def ppeak_cell(s, window, eps=1e-12, sign=1):
    """(k, m) of the arg-max of the periodic AF's Ahat^2 over Omega."""
    s, sv = _s_buf(s)
    w = _win(window)
    pk = np.zeros(2, dtype=np.int64)
    _check(_load().orc_ppeak_cell(_ptr(sv), s.shape[0], int(sign), w.ctypes.data_as(_ip), eps,
                                  pk.ctypes.data_as(_ip)), "ppeak_cell")
    return int(pk[0]), int(pk[1])


def pcell_grad(s, k, m, eps=1e-12, sign=1):
    """(grad_s, grad_phi) of one periodic cell's Ahat^2[k, m]."""
    s, sv = _s_buf(s)
    N = s.shape[0]
    gs = np.zeros(N, dtype=np.complex128)
    gp = np.zeros(N, dtype=np.float64)
    _check(_load().orc_pcell_grad(_ptr(sv), N, int(sign), int(k), int(m), eps, _ptr(gs.view(np.float64)),
                                  _ptr(gp)), "pcell_grad")
    return gs, gp


def pfd_grad_phi(phi, window, w_psl=1.0, w_isl=1.0, beta=50.0, eps=1e-12, sign=1, h=3e-5):
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64))
    w = _win(window)
    g = np.zeros(phi.shape[0], dtype=np.float64)
    _check(_load().orc_pfd_grad_phi(_ptr(phi), phi.shape[0], int(sign), w.ctypes.data_as(_ip), w_psl, w_isl,
                                    beta, eps, h, _ptr(g)), "pfd_grad_phi")
    return g


def optimize_experiment(phi0, window, w_psl, w_isl, beta, eps, spectral_weight, steps, sign=1, lr=1e-2,
                        beta1=0.9, beta2=0.999, adam_eps=1e-8):
    """The experiment of Sec. 7.1 restated: Adam (lr 0.01) on the phases for
    L = L_AF(periodic AF of Eq. 7) + lambda alpha SpectralVariance (Eq. 25);
    per step the loss and dL/dphi of both terms, then one Adam update.
    Returns (phi after `steps` steps, loss before each step)."""
    from . import spectral
    phi = np.asarray(phi0, dtype=np.float64).copy()
    m = np.zeros_like(phi)
    v = np.zeros_like(phi)
    hist = []
    for t in range(1, steps + 1):
        s = signal_from_phase(phi)
        _, gphi, out = pgrad(s, window, w_psl, w_isl, beta, eps, sign)
        sv, _, gsv = spectral.spectral_variance_grad(s)
        hist.append(out[0] + spectral_weight * sv)
        phi, m, v = adam_update(phi, m, v, gphi + spectral_weight * gsv, t, lr, beta1, beta2, adam_eps)
    return phi, np.array(hist)


def match(s, M, window, target, weight=1.0, eps=1e-12, nthreads=None):
    """(sum (Ahat^2 - target)^2, grad_s, grad_phi) of weight * that sum
    (L_match of Eq. 22); target [rows][cols] over the window (box ignored)."""
    s, sv = _s_buf(s)
    w = _win(window)
    N = s.shape[0]
    tg = np.ascontiguousarray(np.asarray(target, dtype=np.float64))
    gs = np.zeros(N, dtype=np.complex128)
    gp = np.zeros(N, dtype=np.float64)
    out = np.zeros(1, dtype=np.float64)
    _check(_load().orc_match(_ptr(sv), N, M, w.ctypes.data_as(_ip), _ptr(tg), weight, eps,
                             _ptr(gs.view(np.float64)), _ptr(gp), _ptr(out), _threads(nthreads)), "match")
    return out[0], gs, gp
