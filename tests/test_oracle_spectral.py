"""Pins for the spectral-variance reference (Sec. 7.1.1, Eq. 25): closed
forms, invariances and finite differences.  CPU only."""
import math

import numpy as np
import pytest

from oracle import spectral
from paper_2506_22935_gb300 import inputs


@pytest.mark.parametrize("N", [8, 16, 64, 256])
def test_flat_and_constant_spectra(N):
    # a Chu sequence has a flat power spectrum: SV = 0
    n = np.arange(N, dtype=np.float64)
    chu = np.exp(-1j * math.pi * n * n / N)
    assert spectral.spectral_variance(chu) < 1e-28
    # s = 1: all power in bin 0, q = (1, 0, ..., 0): SV = (1 - 1/N)/N
    assert abs(spectral.spectral_variance(np.ones(N)) - (1.0 - 1.0 / N) / N) < 1e-15
    # a single impulse has a flat spectrum too
    d = np.zeros(N, dtype=np.complex128)
    d[3] = 2.0 - 1.0j
    assert spectral.spectral_variance(d) < 1e-28


def test_matches_numpy_fft_and_invariances():
    N = 64
    s = inputs.random_complex(7, 1, N)[0].astype(np.complex128)
    P = np.abs(np.fft.fft(s)) ** 2
    sv_np = np.var(P / P.sum())
    sv = spectral.spectral_variance(s)
    assert abs(sv - sv_np) < 1e-15 * max(sv_np, 1e-30) + 1e-20
    # invariant to a global phase, a scale, a circular shift and conjugation
    for t in (np.exp(0.7j) * s, 3.0 * s, np.roll(s, 5), np.conj(s)):
        assert abs(spectral.spectral_variance(t) - sv) < 1e-12 * sv


@pytest.mark.parametrize("N", [8, 32])
def test_gradient_matches_finite_differences(N):
    s = inputs.random_complex(11, 1, N)[0].astype(np.complex128)
    _, gs, _ = spectral.spectral_variance_grad(s)
    h = 1e-6
    fd = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        for unit in (1.0, 1j):
            a, b = s.copy(), s.copy()
            a[i] += h * unit
            b[i] -= h * unit
            fd[i] += unit * (spectral.spectral_variance(a) - spectral.spectral_variance(b)) / (2 * h)
    assert np.linalg.norm(gs - fd) <= 1e-6 * np.linalg.norm(fd)
    phi = inputs.random_phases(12, 1, N)[0].astype(np.float64)
    _, _, gp = spectral.spectral_variance_grad(np.exp(1j * phi))
    fdp = np.zeros(N)
    for i in range(N):
        a, b = phi.copy(), phi.copy()
        a[i] += h
        b[i] -= h
        fdp[i] = (spectral.spectral_variance(np.exp(1j * a)) - spectral.spectral_variance(np.exp(1j * b))) / (2 * h)
    assert np.linalg.norm(gp - fdp) <= 1e-6 * np.linalg.norm(fdp)
    assert abs(gp.sum()) < 1e-12 * np.abs(gp).sum()   # global-phase invariance
