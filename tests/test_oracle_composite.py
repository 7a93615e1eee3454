"""Pins for the mainlobe-width and constant-modulus references (Sec. 5.1,
Eq. 22): closed forms for a rectangular pulse, the autocorrelation against
numpy's correlate, invariances and finite differences.  CPU only."""
import numpy as np
import pytest

from oracle import composite
from paper_2506_22935_gb300 import inputs


def test_autocorrelation_matches_numpy_correlate():
    s = inputs.random_complex(3, 1, 17)[0].astype(np.complex128)
    r = composite.autocorrelation(s)
    # numpy: c[k] = sum_n a[n+k] conj(v[n]); with a = v = s that is r[k]
    ref = np.correlate(s, s, mode="full")
    np.testing.assert_allclose(r, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [4, 16, 64])
@pytest.mark.parametrize("gamma", [5.0, 50.0])
def test_rect_pulse_closed_form(N, gamma):
    # s = 1: r[k] = N - |k|, a2 = (1 - |k|/N)^2
    k = np.arange(-(N - 1), N)
    a2 = (1.0 - np.abs(k) / N) ** 2
    ref = np.sum(np.abs(k) / (1.0 + np.exp(-gamma * (a2 - 0.5))))
    assert abs(composite.mainlobe_width(np.ones(N), gamma) - ref) < 1e-12 * max(ref, 1.0)
    # and the hard -3 dB width is the sharp limit: |k| with a2 > 1/2
    hard = np.sum(np.abs(k)[a2 > 0.5])
    assert abs(composite.mainlobe_width(np.ones(N), 1e6) - hard) < 1e-6 * max(hard, 1.0)


def test_width_invariances():
    s = inputs.random_complex(5, 1, 32)[0].astype(np.complex128)
    w = composite.mainlobe_width(s, 20.0)
    for t in (np.exp(0.3j) * s, 2.5 * s, s[::-1].conj(), np.exp(1j * 0.2 * np.arange(32)) * s):
        assert abs(composite.mainlobe_width(t, 20.0) - w) < 1e-10 * max(w, 1.0)


@pytest.mark.parametrize("gamma", [3.0, 30.0])
def test_width_gradient_matches_finite_differences(gamma):
    N = 16
    # a code with a few near-threshold lags, so the sigmoid is not saturated
    s = inputs.random_complex(7, 1, N)[0].astype(np.complex128) + 0.8
    _, gs, _ = composite.mainlobe_width_grad(s, gamma, 1e-9)
    h = 1e-6
    fd = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        for unit in (1.0, 1j):
            a, b = s.copy(), s.copy()
            a[i] += h * unit
            b[i] -= h * unit
            fd[i] += unit * (composite.mainlobe_width(a, gamma, 1e-9) - composite.mainlobe_width(b, gamma, 1e-9)) / (2 * h)
    assert np.linalg.norm(gs - fd) <= 1e-6 * np.linalg.norm(fd) + 1e-9


def test_modulus_variance_and_gradient():
    N = 24
    assert composite.modulus_variance(np.exp(1j * np.arange(N))) < 1e-30   # constant modulus
    s = inputs.random_complex(9, 1, N)[0].astype(np.complex128)
    a = np.abs(s)
    assert abs(composite.modulus_variance(s) - np.var(a)) < 1e-15
    _, gs = composite.modulus_variance_grad(s)
    h = 1e-6
    fd = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        for unit in (1.0, 1j):
            p, m = s.copy(), s.copy()
            p[i] += h * unit
            m[i] -= h * unit
            fd[i] += unit * (composite.modulus_variance(p) - composite.modulus_variance(m)) / (2 * h)
    assert np.linalg.norm(gs - fd) <= 1e-6 * np.linalg.norm(fd)
