"""Pins for the periodic-AF oracle (the paper's own definition, Sec. 3.1 Eq. 2,
Sec. 4.1 Eq. 7, Algorithm 1): closed forms, identities against the separately
pinned aperiodic oracle, and finite differences.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_22935_gb300 import inputs


def _chu(N, u):
    """Chu sequence exp(-j pi u n^2 / N), N even, u odd: N-periodic, with an
    ideal periodic autocorrelation."""
    n = np.arange(N, dtype=np.float64)
    return np.exp(-1j * math.pi * u * n * n / N)


def _shift_axis(N):
    return np.arange(-(N // 2), N - N // 2)


@pytest.mark.parametrize("N,u", [(16, 1), (16, 3), (32, 5), (64, 7)])
@pytest.mark.parametrize("sign", [1, -1])
def test_chu_closed_form(N, u, sign):
    """s[n] conj(s[n-k]) = exp(j pi u k^2/N) exp(-j 2 pi u k n / N), so
    |X[k,m]| = N where m = sign*u*k (mod N) and 0 elsewhere: a ridge whose
    slope also fixes the sign of the Doppler exponent."""
    X = oracle.paf_complex(_chu(N, u), sign)
    k = _shift_axis(N)[:, None]
    m = _shift_axis(N)[None, :]
    on = ((m - sign * u * k) % N) == 0
    np.testing.assert_allclose(np.abs(X[on]), N, rtol=0, atol=1e-9 * N)
    np.testing.assert_allclose(np.abs(X[~on]), 0.0, rtol=0, atol=1e-9 * N)


@pytest.mark.parametrize("N", [8, 16, 24])
def test_periodic_equals_sum_of_two_aperiodic_rows(N):
    """For 0 <= k < N, s[(n-k) mod N] is s[n-k] for n >= k and s[n-k+N] for
    n < k, so the periodic row k is the aperiodic row k plus the aperiodic row
    k - N, both transformed with M = N points and the -j sign of the
    aperiodic definition."""
    s = inputs.random_complex(5, 1, N)[0].astype(np.complex128)
    Xp = oracle.paf_complex(s, -1)
    Xa = oracle.af_complex(s, N, -(N - 1), N - 1, -(N // 2), N - 1 - N // 2)  # rows k = -(N-1)..N-1
    for i, k in enumerate(_shift_axis(N)):
        kp = k if k >= 0 else k + N          # periodic row index in [0, N)
        a = Xa[kp + (N - 1)]
        b = Xa[kp - N + (N - 1)] if kp > 0 else 0.0
        np.testing.assert_allclose(Xp[i], a + b, rtol=0, atol=1e-11 * N * N)


def test_origin_parseval_symmetry_and_sign():
    N = 32
    s = inputs.random_complex(9, 1, N)[0].astype(np.complex128)
    E = oracle.energy(s)
    Xp = oracle.paf_complex(s, 1)
    Xm = oracle.paf_complex(s, -1)
    c = N // 2
    assert abs(Xp[c, c] - E) < 1e-11 * E                      # X[0,0] = E
    assert np.abs(Xp).max() <= E * (1 + 1e-12)                # Cauchy-Schwarz
    a2 = np.abs(s) ** 2
    for i, k in enumerate(_shift_axis(N)):                    # per-row Parseval
        rhs = N * np.sum(a2 * np.roll(a2, k))
        assert abs(np.sum(np.abs(Xp[i]) ** 2) - rhs) < 1e-10 * rhs
    # |X[-k, m]| = |X[k, -m]| (indices mod N) and the sign flip X+[k,m] = X-[k,-m]
    idx = lambda v: (v + c) % N
    for k in range(-c, c):
        for m in range(-c, c):
            assert abs(abs(Xp[idx(-k), idx(m)]) - abs(Xp[idx(k), idx(-m)])) < 1e-10 * E
            assert abs(Xp[idx(k), idx(m)] - Xm[idx(k), idx(-m)]) < 1e-10 * E


def test_chi_normalised_is_chi_over_max():
    s = inputs.random_complex(3, 1, 16)[0].astype(np.complex128)
    chi = oracle.paf_chi(s, 1, normalise=False)
    chin = oracle.paf_chi(s, 1, normalise=True)
    np.testing.assert_allclose(chin, chi / chi.max(), rtol=1e-12)


@pytest.mark.parametrize("window,lp", [
    ((-8, 7, -8, 7, 0, 0), (1.0, 1.0, 20.0)),
    ((-3, 5, -4, 6, 0, 1), (0.5, 1.0, 50.0)),
    ((-8, 7, -8, 7, -1, -1), (0.0, 1.0, 50.0)),
    ((2, 6, -8, 7, 0, 0), (1.0, 0.0, 30.0)),
])
@pytest.mark.parametrize("sign", [1, -1])
def test_periodic_gradient_matches_finite_differences(window, lp, sign):
    N = 16
    phi = inputs.random_phases(21, 1, N)[0].astype(np.float64)
    s = np.exp(1j * phi)
    gs, gp, out = oracle.pgrad(s, window, *lp, 1e-12, sign)
    fd = oracle.pfd_grad_phi(phi, window, *lp, 1e-12, sign)
    # (a full-window ISL has an exactly zero phase gradient: the FD noise floor is ~1e-9)
    assert np.linalg.norm(gp - fd) <= 1e-7 * np.linalg.norm(fd) + 1e-8
    # complex input: central differences of the loss in Re s and Im s
    z = inputs.random_complex(22, 1, N)[0].astype(np.complex128)
    gz, _, _ = oracle.pgrad(z, window, *lp, 1e-12, sign)
    h = 3e-6
    fdz = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        for part, unit in ((0, 1.0), (1, 1j)):
            zp, zm = z.copy(), z.copy()
            zp[i] += h * unit
            zm[i] -= h * unit
            d = (oracle.ploss(zp, window, *lp, 1e-12, sign)[0] - oracle.ploss(zm, window, *lp, 1e-12, sign)[0]) / (2 * h)
            fdz[i] += d * unit
    assert np.linalg.norm(gz - fdz) <= 1e-6 * np.linalg.norm(fdz) + 5e-8


def test_periodic_phase_gradient_is_global_phase_invariant():
    N = 32
    phi = inputs.random_phases(23, 1, N)[0].astype(np.float64)
    _, gp, _ = oracle.pgrad(np.exp(1j * phi), oracle.full_pwindow(N), 1.0, 1.0, 50.0, 1e-12, 1)
    assert abs(gp.sum()) < 1e-10 * np.abs(gp).sum()
