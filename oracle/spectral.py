"""FP64 reference of the spectral-variance term of the paper's experiment
loss (Sec. 7.1.1, Eq. 25): SpectralVariance = var{|FFT(s)|^2 / sum |FFT(s)|^2}
(population variance over the N bins), and its gradient.  Test
infrastructure: only tests, smoke and the bench's reference legs use it.

Every sum is a direct sum over an explicit DFT matrix (no FFT), written from
the definitions:
    S[f]  = sum_n s[n] exp(-j 2 pi f n / N)
    P[f]  = |S[f]|^2,  q = P / sum P
    SV    = (1/N) sum_f (q[f] - 1/N)^2
Gradient (Wirtinger; P[f] = S[f] conj(S[f]) and conj(S[f]) carries s*[n] with
the factor exp(+j 2 pi f n / N)):
    dSV/dq[f]   = (2/N) (q[f] - 1/N)
    dSV/dP[g]   = (dSV/dq[g] - sum_f q[f] dSV/dq[f]) / sum P
    dSV/ds*[n]  = sum_g dSV/dP[g] S[g] exp(+j 2 pi g n / N)
exported as grad_s = 2 dSV/ds* and, for s = exp(j phi), grad_phi =
2 Im(dSV/ds* conj(s)), the conventions of the AF gradient.
"""
from __future__ import annotations

import numpy as np


def _dft_matrix(N: int) -> np.ndarray:
    f = np.arange(N)[:, None]
    n = np.arange(N)[None, :]
    return np.exp(-2j * np.pi * ((f * n) % N) / N)


def spectral_variance(s) -> float:
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    S = _dft_matrix(N) @ s
    P = np.abs(S) ** 2
    q = P / P.sum()
    return float(np.mean((q - 1.0 / N) ** 2))


def spectral_variance_grad(s):
    """(SV, grad_s = 2 dSV/ds*, grad_phi = 2 Im(dSV/ds* conj(s)))."""
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    F = _dft_matrix(N)
    S = F @ s
    P = np.abs(S) ** 2
    tot = P.sum()
    q = P / tot
    sv = float(np.mean((q - 1.0 / N) ** 2))
    dq = (2.0 / N) * (q - 1.0 / N)
    dP = (dq - np.sum(q * dq)) / tot
    g = np.conj(F).T @ (dP * S)          # sum_g dP[g] S[g] exp(+j 2 pi g n / N)
    return sv, 2.0 * g, 2.0 * np.imag(g * np.conj(s))
