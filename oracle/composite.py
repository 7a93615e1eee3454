"""FP64 reference of two terms of the paper's composite loss (Sec. 5.1,
Sec. 5.2 Eq. 22): the differentiable mainlobe width and the constant-modulus
penalty.  Test infrastructure: only tests, smoke and the bench's reference
legs use it.

Definitions (direct sums, no FFT):
    r[k]   = sum_n s[n] conj(s[n-k])         zero-Doppler column of the AF
             (Eq. 8 summed over n, aperiodic, k = -(N-1)..N-1)
    a2[k]  = (|r[k]|^2 + eps) / E^2,  E = sum |s|^2   (chi(k,0) / chi(0,0))
    W      = sum_k |k| sigmoid(gamma (a2[k] - 1/2))   (the sigmoid form of the
             -3 dB mainlobe width, Sec. 5.1)
    V      = var(|s|) = (1/N) sum_n (|s[n]| - mean |s|)^2    (L_const, Eq. 22)
Gradients (Wirtinger, exported as 2 dL/ds* like the AF gradient):
    dW/da2[k] = |k| gamma sig (1 - sig)
    G[k] = dW/dr*[k] = dW/da2[k] r[k] / E^2;  r*[k] carries s*[n] (with the
    factor s[n-k]) and r[k] carries s*[n-k] (with the factor s[n]), so the
    product rule adds G[k] s[n-k] at n and conj(G[k]) s[n] at n-k, plus the
    energy term dW/dE = -(2/E) sum_k dW/da2[k] a2[k], dE/ds* = s;
    dV/ds*[n] = (|s[n]| - mean) s[n] / (N |s[n]|)   (0 where s[n] = 0).
"""
from __future__ import annotations

import numpy as np


def autocorrelation(s) -> np.ndarray:
    """r[k] for k = -(N-1)..N-1 (index k + N - 1)."""
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    r = np.zeros(2 * N - 1, dtype=np.complex128)
    for k in range(-(N - 1), N):
        acc = 0.0j
        for n in range(max(0, k), min(N, N + k)):
            acc += s[n] * np.conj(s[n - k])
        r[k + N - 1] = acc
    return r


def _sig(x):
    """Logistic sigmoid, evaluated without overflow for large |x|."""
    x = np.asarray(x, dtype=np.float64)
    e = np.exp(-np.abs(x))
    return np.where(x >= 0, 1.0 / (1.0 + e), e / (1.0 + e))


def mainlobe_width(s, gamma=50.0, eps=0.0) -> float:
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    E = np.sum(np.abs(s) ** 2)
    r = autocorrelation(s)
    a2 = (np.abs(r) ** 2 + eps) / E ** 2
    k = np.arange(-(N - 1), N)
    return float(np.sum(np.abs(k) * _sig(gamma * (a2 - 0.5))))


def mainlobe_width_grad(s, gamma=50.0, eps=0.0):
    """(W, grad_s = 2 dW/ds*, grad_phi = 2 Im(dW/ds* conj(s)))."""
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    E = np.sum(np.abs(s) ** 2)
    r = autocorrelation(s)
    a2 = (np.abs(r) ** 2 + eps) / E ** 2
    k = np.arange(-(N - 1), N)
    sg = _sig(gamma * (a2 - 0.5))
    W = float(np.sum(np.abs(k) * sg))
    dWda2 = np.abs(k) * gamma * sg * (1.0 - sg)
    G = dWda2 * r / E ** 2                       # dW/dr*[k]
    g = np.zeros(N, dtype=np.complex128)
    for i, kk in enumerate(k):
        for n in range(max(0, kk), min(N, N + kk)):
            # r[k] = sum_n s[n] conj(s[n-k]): r*[k] carries s*[n] (factor s[n-k]),
            # r[k] carries s*[n-k] (factor s[n]); L real, so dL/dr = conj(G)
            g[n] += G[i] * s[n - kk]
            g[n - kk] += np.conj(G[i]) * s[n]
    g += -(2.0 / E) * np.sum(dWda2 * a2) * s
    return W, 2.0 * g, 2.0 * np.imag(g * np.conj(s))


def modulus_variance(s) -> float:
    a = np.abs(np.asarray(s, dtype=np.complex128))
    return float(np.mean((a - a.mean()) ** 2))


def modulus_variance_grad(s):
    s = np.asarray(s, dtype=np.complex128)
    N = s.shape[0]
    a = np.abs(s)
    V = float(np.mean((a - a.mean()) ** 2))
    unit = np.where(a > 0, s / np.where(a > 0, a, 1.0), 0.0)
    g = (a - a.mean()) * unit / N
    return V, 2.0 * g
