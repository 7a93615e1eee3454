"""Pins for the oracle's hard PSL (Eq. 18: the maximum of Ahat^2 over the
sidelobe region, with the subgradient through one arg-max cell; selected by
beta = inf): closed forms of the rectangular pulse and the Chu sequence, the
arg-max rule on exact ties, an independent product-rule derivation of one
cell's gradient (which involves only the arg-max delay row), mirror cells,
finite differences away from ties, and the beta -> infinity limit of the
log-sum-exp PSL.  CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2506_22935_gb300 import inputs

INF = math.inf


def _dirichlet2(L, x):
    """sin^2(pi L x) / sin^2(pi x), with the limit L^2 at integer x."""
    den = np.sin(np.pi * x)
    if abs(x - round(x)) < 1e-12:
        return float(L * L)
    return float((np.sin(np.pi * L * x) / den) ** 2)


@pytest.mark.parametrize("N,M", [(8, 16), (16, 64), (13, 32)])
def test_rect_pulse_hard_psl_closed_form(N, M):
    """s = 1 and eps = 0: Ahat^2[k,m] = sin^2(pi m (N-|k|)/M) / (N^2 sin^2(pi m/M)),
    whose largest value off the zero-delay mainlobe is ((N-1)/N)^2 at
    (k, m) = (+-1, 0); the first in row-major order is (-1, 0).  ISL over Omega
    is M (the volume identity) minus the box cells (0, |m| <= M/N - 1)."""
    s = np.ones(N, dtype=np.complex128)
    box = M // N - 1
    win = (-(N - 1), N - 1, -(M // 2), M - 1 - M // 2, 0, box)
    out = orc.loss(s, M, win, 0.7, 0.3, INF, 0.0)
    psl = ((N - 1) / N) ** 2
    isl = M - sum(_dirichlet2(N, m / M) for m in range(-box, box + 1)) / N ** 2
    assert abs(out[1] - psl) < 1e-12 and abs(out[3] - psl) < 1e-12 and abs(out[6] - psl) < 1e-12
    assert abs(out[2] - isl) < 1e-9 * M
    assert abs(out[0] - (0.7 * psl + 0.3 * isl)) < 1e-9 * M
    assert orc.peak_cell(s, M, win, 0.0) == (-1, 0)


@pytest.mark.parametrize("N,u", [(16, 1), (16, 3), (32, 5)])
def test_chu_periodic_hard_psl_ties(N, u):
    """Chu sequence exp(-j pi u n^2 / N) with sign +1: |X[k,m]| = N on the
    ridge m = u k (mod N), 0 elsewhere, so the hard PSL over every cell but the
    origin is exactly 1, reached at every ridge cell k != 0.  The arg-max rule
    takes the first in row-major order: k = -N/2, m = -u N/2 mod N in
    [-N/2, N/2)."""
    n = np.arange(N, dtype=np.float64)
    s = np.exp(-1j * math.pi * u * n * n / N)
    win = orc.full_pwindow(N)
    out = orc.ploss(s, win, 1.0, 0.0, INF, 0.0, sign=1)
    assert abs(out[1] - 1.0) < 1e-12 and abs(out[3] - 1.0) < 1e-12
    k0 = -(N // 2)
    m0 = ((u * k0 + N // 2) % N) - N // 2
    assert orc.ppeak_cell(s, win, 0.0, sign=1) == (k0, m0)
    gs, gp, _ = orc.pgrad(s, win, 1.0, 0.0, INF, 0.0, sign=1)
    cs, cp = orc.pcell_grad(s, k0, m0, 0.0, sign=1)
    np.testing.assert_allclose(gs, cs, atol=1e-12)


def _cell_grad_direct(s, M, k, m, eps):
    """d Ahat^2[k,m] / d s* by the product rule on the single sum
    X = sum_n s[n] conj(s[n-k]) w^(m n), w = exp(-2 pi j / M), written here
    directly: dX/ds*[p] = s[p+k] w^(m (p+k)), d conj(X)/ds*[p] = s[p-k] conj(w^(m p)),
    d|X|^2/ds* = X d conj(X)/ds* + conj(X) dX/ds*, and d(1/E^2)/ds* = -2 s / E^3.
    Only delay row k enters.  Returns 2 dAhat^2/ds* (the exported convention)."""
    N = len(s)
    n = np.arange(N)
    lag = np.zeros(N, dtype=np.complex128)
    ok = (n - k >= 0) & (n - k < N)
    lag[ok] = np.conj(s[n[ok] - k])
    X = np.sum(s * lag * np.exp(-2j * np.pi * ((m * n) % M) / M))
    E = float(np.sum(np.abs(s) ** 2))
    a2 = (abs(X) ** 2 + eps) / E ** 2
    d = np.zeros(N, dtype=np.complex128)
    for p in range(N):
        if 0 <= p + k < N:
            d[p] += np.conj(X) * s[p + k] * np.exp(-2j * np.pi * ((m * (p + k)) % M) / M)
        if 0 <= p - k < N:
            d[p] += X * s[p - k] * np.exp(2j * np.pi * ((m * p) % M) / M)
    return 2.0 * (d / E ** 2 - 2.0 * a2 / E * s)


@pytest.mark.parametrize("N,M,k,m", [(9, 32, 3, 5), (16, 32, -7, -16), (12, 64, 0, 9), (7, 16, 6, -3)])
def test_cell_grad_matches_direct_product_rule(N, M, k, m):
    s = inputs.random_complex(41 + N, 1, N)[0].astype(np.complex128)
    gs, gp = orc.cell_grad(s, M, k, m, 1e-3)
    want = _cell_grad_direct(s, M, k, m, 1e-3)
    np.testing.assert_allclose(gs, want, atol=1e-12 * np.abs(want).max())
    # phase gradient of the same cell: Im(conj(grad_s) j s) = dAhat^2/dphi
    np.testing.assert_allclose(gp, np.real(np.conj(gs) * 1j * s), atol=1e-12 * np.abs(want).max())


def test_mirror_cells_have_equal_gradients():
    """|X[-k,-m]| = |X[k,m]| for every s: the two cells are one function of s,
    so a tie between mirror cells leaves the hard-PSL gradient unique."""
    N, M = 11, 32
    s = inputs.random_complex(5, 1, N)[0].astype(np.complex128)
    for k, m in [(3, 5), (1, -16), (0, 7)]:
        mm = -m if m != -(M // 2) else m
        a, _ = orc.cell_grad(s, M, k, m, 1e-6)
        b, _ = orc.cell_grad(s, M, -k, mm, 1e-6)
        np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())


def _gap(s, M, win, eps):
    """Largest Ahat^2 over Omega minus the largest among cells that are neither
    the arg-max nor its mirror."""
    A = orc.af_ahat(s, M, win[0], win[1], win[2], win[3], eps) ** 2
    ks = np.arange(win[0], win[1] + 1)[:, None]
    ms = np.arange(win[2], win[3] + 1)[None, :]
    omega = ~((np.abs(ks) <= win[4]) & (np.abs(ms) <= win[5]))
    A = np.where(omega, A, -np.inf)
    pk, pm = orc.peak_cell(s, M, win, eps)
    mm = -pm if pm != -(M // 2) else pm
    top = A[pk - win[0], pm - win[2]]
    A[pk - win[0], pm - win[2]] = -np.inf
    if win[0] <= -pk <= win[1] and win[2] <= mm <= win[3]:
        A[-pk - win[0], mm - win[2]] = -np.inf
    return top - A.max()


@pytest.mark.parametrize("N,M,win", [
    (10, 32, None),
    (9, 16, (-8, 8, -8, 7, 0, 1)),
    (12, 32, (-5, 7, -9, 12, 0, 0)),
])
@pytest.mark.parametrize("kind", ["phase", "complex"])
def test_hard_psl_gradient_against_finite_differences(N, M, win, kind):
    """Away from ties the hard maximum is differentiable: the oracle's
    gradient (arg-max cell plus the ISL term and the energy term) matches
    central differences of its own loss."""
    win = win or orc.full_window(N, M)
    for seed in range(20):
        if kind == "phase":
            phi = inputs.random_phases(300 + seed, 1, N)[0].astype(np.float64)
            s = orc.signal_from_phase(phi)
        else:
            s = inputs.random_complex(300 + seed, 1, N)[0].astype(np.complex128)
        if _gap(s, M, win, 1e-12) > 1e-3:
            break
    else:
        pytest.skip("no input with a clear peak")
    gs, gp, out = orc.grad(s, M, win, 1.0, 0.5, INF, 1e-12)
    if kind == "phase":
        fd = orc.fd_grad_phi(phi, M, win, 1.0, 0.5, INF, 1e-12, h=1e-6)
        np.testing.assert_allclose(gp, fd, atol=1e-7 * max(1.0, np.abs(fd).max()))
    else:
        fd = orc.fd_grad_s(s, M, win, 1.0, 0.5, INF, 1e-12, h=1e-6)
        np.testing.assert_allclose(gs, fd, atol=1e-7 * max(1.0, np.abs(fd).max()))
    # the PSL part is exactly the arg-max cell's gradient
    g_isl, _, _ = orc.grad(s, M, win, 0.0, 0.5, INF, 1e-12)
    g_cell, _ = orc.cell_grad(s, M, *orc.peak_cell(s, M, win, 1e-12), 1e-12)
    np.testing.assert_allclose(gs - g_isl, g_cell, atol=1e-12 * np.abs(g_cell).max())


def test_periodic_hard_psl_against_finite_differences():
    N = 16
    win = orc.full_pwindow(N)
    phi = inputs.random_phases(77, 1, N)[0].astype(np.float64)
    s = orc.signal_from_phase(phi)
    _, gp, out = orc.pgrad(s, win, 1.0, 0.25, INF, 1e-12, sign=1)
    fd = orc.pfd_grad_phi(phi, win, 1.0, 0.25, INF, 1e-12, sign=1, h=1e-6)
    np.testing.assert_allclose(gp, fd, atol=1e-7 * np.abs(fd).max())
    k, m = orc.ppeak_cell(s, win, 1e-12, sign=1)
    _, cp = orc.pcell_grad(s, k, m, 1e-12, sign=1)
    _, gi, _ = orc.pgrad(s, win, 0.0, 0.25, INF, 1e-12, sign=1)
    np.testing.assert_allclose(gp - gi, cp, atol=1e-12 * np.abs(cp).max())


def test_soft_psl_tends_to_the_hard_psl():
    """PSL_soft lies in [PSL_hard, PSL_hard + log|Omega|/beta] and, with a clear
    peak, its gradient tends to the arg-max cell's as beta grows."""
    N, M = 10, 32
    win = orc.full_window(N, M)
    s = orc.signal_from_phase(inputs.random_phases(303, 1, N)[0].astype(np.float64))
    hard = orc.loss(s, M, win, 1.0, 0.0, INF)
    gh, _, _ = orc.grad(s, M, win, 1.0, 0.0, INF)
    for beta in (1e3, 1e4):
        soft = orc.loss(s, M, win, 1.0, 0.0, beta)
        assert hard[3] <= soft[1] <= hard[3] + math.log(soft[5]) / beta + 1e-15
    gsoft, _, _ = orc.grad(s, M, win, 1.0, 0.0, 2e4)
    assert np.linalg.norm(gsoft - gh) <= 1e-6 * np.linalg.norm(gh)
