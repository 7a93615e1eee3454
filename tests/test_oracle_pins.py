"""Pins for the FP64 oracle against facts that do not come from the oracle:
closed forms, identities, a textbook sequence, statistics and finite
differences.  Each test names the fact it uses; together they catch a dropped
term, a wrong sign or index, a transposed operand, a wrong support or a wrong
normaliser anywhere in the oracle.  CPU only."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2506_22935_gb300 import inputs


def _all(N, M):
    return -(N - 1), N - 1, -(M // 2), M - 1 - M // 2


def _grid(N, M):
    k_lo, k_hi, m_lo, m_hi = _all(N, M)
    k = np.arange(k_lo, k_hi + 1)[:, None]
    m = np.arange(m_lo, m_hi + 1)[None, :]
    return k, m


def _dirichlet(L, x):
    """|sin(pi L x) / sin(pi x)|, with the limit L at integer x."""
    x, L = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(L, dtype=np.float64))
    den = np.sin(np.pi * x)
    near = np.abs(x - np.rint(x)) < 1e-12
    out = np.where(near, L, np.abs(np.sin(np.pi * L * x) / np.where(near, 1.0, den)))
    return out


@pytest.mark.parametrize("N,M", [(1, 8), (5, 8), (16, 32), (16, 16), (13, 64), (31, 64)])
def test_rect_pulse_closed_form(N, M):
    """s = 1: |X[k,m]| = |sin(pi m (N-|k|)/M) / sin(pi m / M)|, and N-|k| at
    m = 0 (the aperiodic lag product has N-|k| ones; Eq. 8, Eq. 11)."""
    s = np.ones(N, dtype=np.complex128)
    X = orc.af_complex(s, M, *_all(N, M))
    k, m = _grid(N, M)
    want = _dirichlet(N - np.abs(k), m / M)
    np.testing.assert_allclose(np.abs(X), want, rtol=0, atol=1e-10 * N)


@pytest.mark.parametrize("N,M", [(64, 128), (16, 64), (32, 32)])
def test_lfm_closed_form(N, M):
    """Discrete chirp phi = pi n^2 / N: R[k,n] = exp(j pi (2 n k - k^2)/N), so
    |X[k,m]| = |sin(pi (N-|k|) x) / sin(pi x)| with x = k/N - m/M: a ridge at
    m = k M / N.  A flipped DFT sign or a conjugate on the wrong factor of the
    lag product moves the ridge to m = -k M / N and fails this."""
    n = np.arange(N, dtype=np.float64)
    s = np.exp(1j * np.pi * n * n / N)
    X = orc.af_complex(s, M, *_all(N, M))
    k, m = _grid(N, M)
    want = _dirichlet(N - np.abs(k), k / N - m / M)
    np.testing.assert_allclose(np.abs(X), want, rtol=0, atol=1e-9 * N)


def test_zero_delay_zero_doppler_is_energy():
    """X[0,0] = sum |s|^2 = E exactly, and max |X| = E (Cauchy-Schwarz; the
    energy normaliser equals the max normaliser of Eq. 17)."""
    s = inputs.random_complex(11, 1, 37)[0].astype(np.complex128)
    M = 128
    X = orc.af_complex(s, M, *_all(37, M))
    E = float(np.sum(np.abs(s) ** 2))
    assert abs(X[36, 64] - E) < 1e-12 * E
    assert np.max(np.abs(X)) <= E * (1 + 1e-12)
    assert abs(orc.energy(s) - E) < 1e-12 * E


def test_unit_modulus_zero_delay_row_is_phase_free():
    """For |s| = 1 the k = 0 row is R[0,n] = 1: |X[0,m]| = |sin(pi m N/M)/sin(pi m/M)|
    whatever the phases."""
    N, M = 24, 64
    phi = inputs.random_phases(3, 1, N)[0].astype(np.float64)
    s = orc.signal_from_phase(phi)
    row = orc.af_complex(s, M, 0, 0, -(M // 2), M // 2 - 1)[0]
    m = np.arange(-(M // 2), M // 2)
    np.testing.assert_allclose(np.abs(row), _dirichlet(N, m / M), atol=1e-11)


def test_symmetry_negative_delay_doppler():
    """|X[-k,-m]| = |X[k,m]| for any s (substitute n -> n + k)."""
    N, M = 19, 64
    s = inputs.random_complex(5, 1, N)[0].astype(np.complex128)
    X = np.abs(orc.af_complex(s, M, *_all(N, M)))
    # rows k -> -k; columns m -> -m (column of m=-M/2 maps to itself mod M)
    k_idx = np.arange(2 * N - 1)
    m_vals = np.arange(-(M // 2), M // 2)
    col_of_neg = ((-m_vals + M // 2) % M)
    np.testing.assert_allclose(X[::-1][:, col_of_neg], X, rtol=1e-12, atol=1e-12)
    assert k_idx.size == X.shape[0]


@pytest.mark.parametrize("N,M", [(13, 16), (13, 32), (8, 8), (20, 64)])
def test_parseval_rows_and_volume(N, M):
    """Per row (M >= N): sum_m |X[k,m]|^2 = M sum_n |s[n]|^2 |s[n-k]|^2, and in
    total the discrete volume identity sum_{k,m} |X|^2 = M E^2."""
    s = inputs.random_complex(7, 1, N)[0].astype(np.complex128)
    X = orc.af_complex(s, M, *_all(N, M))
    a2 = np.abs(s) ** 2
    for i, k in enumerate(range(-(N - 1), N)):
        n = np.arange(max(0, k), min(N, N + k))
        want = M * np.sum(a2[n] * a2[n - k])
        assert abs(np.sum(np.abs(X[i]) ** 2) - want) <= 1e-11 * M * np.sum(a2) ** 2
    E = np.sum(a2)
    assert abs(np.sum(np.abs(X) ** 2) - M * E * E) <= 1e-11 * M * E * E


@pytest.mark.parametrize("M", [16, 32, 64])
def test_barker13(M):
    """Barker-13: zero-Doppler aperiodic sidelobes |X[k,0]| <= 1 (k != 0) and
    X[0,0] = 13 (the textbook defining property of Barker codes)."""
    s = inputs.barker13().astype(np.complex128)
    X = orc.af_complex(s, M, -12, 12, 0, 0)[:, 0]
    assert abs(X[12] - 13) < 1e-12
    side = np.abs(np.delete(X, 12))
    assert np.all(side <= 1 + 1e-12)
    # the sidelobes of a Barker code alternate between 0 and 1 in magnitude
    assert set(np.rint(side).astype(int)) <= {0, 1}


def test_random_phase_mean_power():
    """For i.i.d. uniform phases, E|X[k,m]|^2 = N - |k| for k != 0 (the N-|k|
    unit-modulus terms are pairwise uncorrelated)."""
    N, M, B = 16, 32, 400
    phis = inputs.random_phases(21, B, N).astype(np.float64)
    acc = np.zeros((2 * N - 1, M))
    for b in range(B):
        X = orc.af_complex(orc.signal_from_phase(phis[b]), M, *_all(N, M), nthreads=1)
        acc += np.abs(X) ** 2
    acc /= B
    k = np.arange(-(N - 1), N)
    for i, kk in enumerate(k):
        if kk == 0:
            continue
        mean = acc[i].mean()
        assert abs(mean - (N - abs(kk))) < 0.08 * (N - abs(kk)) + 0.05


def test_ahat_normalisation_and_eps():
    """Ahat = sqrt(|X|^2 + eps)/E: 1 at the origin with eps = 0, and the eps
    term adds exactly eps/E^2 to every Ahat^2."""
    N, M = 9, 32
    s = inputs.random_complex(13, 1, N)[0].astype(np.complex128)
    E = float(np.sum(np.abs(s) ** 2))
    A0 = orc.af_ahat(s, M, *_all(N, M), eps=0.0)
    A1 = orc.af_ahat(s, M, *_all(N, M), eps=0.25)
    assert abs(A0[N - 1, M // 2] - 1.0) < 1e-13
    np.testing.assert_allclose(A1 ** 2 - A0 ** 2, 0.25 / E ** 2, rtol=1e-9, atol=1e-15)
    cells = orc.af_cells(s, M, [0, 3, -5, 8], [0, -16, 15, 7], 0.25)
    k_lo, _, m_lo, _ = _all(N, M)
    want = [A1[k - k_lo, m - m_lo] for k, m in [(0, 0), (3, -16), (-5, 15), (8, 7)]]
    np.testing.assert_allclose(cells, want, rtol=1e-13)


def test_isl_volume_closed_form():
    """ISL over every cell = sum Ahat^2 = (M E^2 + eps * cells) / E^2 (volume
    identity); excluding only the origin removes exactly (E^2 + eps)/E^2."""
    N, M, eps = 12, 32, 1e-3
    s = inputs.random_complex(17, 1, N)[0].astype(np.complex128)
    E = float(np.sum(np.abs(s) ** 2))
    cells = (2 * N - 1) * M
    out = orc.loss(s, M, (*_all(N, M), -1, -1), 0.0, 1.0, 10.0, eps)
    assert abs(out[2] - (M + eps * cells / E ** 2)) < 1e-10 * M
    assert out[5] == cells
    out0 = orc.loss(s, M, (*_all(N, M), 0, 0), 0.0, 1.0, 10.0, eps)
    assert abs(out0[2] - (M + eps * cells / E ** 2 - (E ** 2 + eps) / E ** 2)) < 1e-10 * M
    assert out0[5] == cells - 1
    assert abs(out0[0] - out0[2]) < 1e-14 * M and abs(out0[4] - E) < 1e-12 * E


def test_psl_on_rect_pulse_zeros():
    """Rect pulse N=4, M=8, row k=0: |X[0,m]| = |sin(pi m/2)/sin(pi m/8)| is 0 at
    m = -4, -2, 2 and 1/sin(3 pi/8) at m = +-3.  With the box |m|<=1 excluded,
    Omega = {-4,-3,-2,2,3}: ISL = 2a, PSL_hard = a, PSL_soft =
    log(3 + 2 exp(beta a))/beta with a = 1/(16 sin^2(3 pi/8))."""
    s = np.ones(4, dtype=np.complex128)
    a = 1.0 / (16.0 * math.sin(3 * math.pi / 8) ** 2)
    for beta in (0.5, 50.0, 5000.0):
        out = orc.loss(s, 8, (0, 0, -4, 3, 0, 1), 1.0, 0.0, beta, 0.0)
        assert abs(out[2] - 2 * a) < 1e-14
        assert abs(out[3] - a) < 1e-14
        want = a + math.log(2.0 + 3.0 * math.exp(-beta * a)) / beta
        assert abs(out[1] - want) < 1e-13
        assert out[5] == 5
    # large beta: soft max -> hard max + log(#ties)/beta
    out = orc.loss(s, 8, (0, 0, -4, 3, 0, 1), 1.0, 0.0, 1e6, 0.0)
    assert abs(out[1] - (a + math.log(2.0) / 1e6)) < 1e-12


FD_CASES = [
    # N, M, window(6) or None (full), w_psl, w_isl, beta
    (1, 8, None, 1.0, 1.0, 50.0),
    (2, 8, None, 1.0, 1.0, 50.0),
    (3, 8, None, 0.0, 1.0, 5.0),
    (5, 16, None, 1.0, 0.0, 50.0),
    (5, 8, (-2, 3, -3, 2, 0, 0), 1.0, 1.0, 20.0),
    (13, 32, None, 1.0, 1.0, 50.0),
    (16, 16, (-4, 9, -8, 7, 1, 2), 0.7, 0.3, 30.0),
    (13, 64, (0, 12, -10, 31, 0, 0), 1.0, 1.0, 50.0),
]


def _win(N, M, w):
    return orc.full_window(N, M) if w is None else w


@pytest.mark.parametrize("N,M,w,w_psl,w_isl,beta", FD_CASES)
def test_adjoint_phase_matches_finite_differences(N, M, w, w_psl, w_isl, beta):
    """dL/dphi of the Wirtinger adjoint (Eqs. 13-15) against FP64 central
    differences of the loss itself."""
    phi = inputs.random_phases(100 + N, 1, N)[0].astype(np.float64)
    win = _win(N, M, w)
    s = orc.signal_from_phase(phi)
    _, gphi, _ = orc.grad(s, M, win, w_psl, w_isl, beta, 1e-12)
    fd = orc.fd_grad_phi(phi, M, win, w_psl, w_isl, beta, 1e-12, h=3e-5)
    scale = max(np.linalg.norm(fd), 1e-6)
    assert np.linalg.norm(gphi - fd) <= 1e-7 * scale + 1e-9


@pytest.mark.parametrize("N,M,w,w_psl,w_isl,beta", FD_CASES)
def test_adjoint_complex_matches_finite_differences(N, M, w, w_psl, w_isl, beta):
    """2 dL/ds* = dL/dRe s + j dL/dIm s for general complex s (this includes the
    energy-normaliser term, which vanishes for unit-modulus input)."""
    s = inputs.random_complex(200 + N, 1, N)[0].astype(np.complex128)
    win = _win(N, M, w)
    gs, _, _ = orc.grad(s, M, win, w_psl, w_isl, beta, 1e-9)
    fd = orc.fd_grad_s(s, M, win, w_psl, w_isl, beta, 1e-9, h=3e-5)
    scale = max(np.linalg.norm(fd), 1e-6)
    assert np.linalg.norm(gs - fd) <= 1e-7 * scale + 1e-9


def test_global_phase_invariance_and_zero_row():
    """L(phi + c) = L(phi), so sum_p dL/dphi[p] = 0; a loss that only sees the
    k = 0 row of a unit-modulus code is constant, so its gradient is 0."""
    N, M = 20, 64
    phi = inputs.random_phases(31, 1, N)[0].astype(np.float64)
    s = orc.signal_from_phase(phi)
    _, g, _ = orc.grad(s, M, orc.full_window(N, M), 1.0, 1.0, 50.0, 1e-12)
    assert abs(g.sum()) < 1e-11 * max(1.0, np.abs(g).sum())
    assert np.abs(g).max() > 1e-4
    _, g0, _ = orc.grad(s, M, (0, 0, -32, 31, 0, 1), 1.0, 1.0, 50.0, 1e-12)
    assert np.abs(g0).max() < 1e-12


def test_phase_gradient_is_projection_of_complex_gradient():
    """For s = exp(j phi), dL/dphi = Re(conj(grad_s) * j s) (chain rule through
    ds/dphi = j s), tying the two exported gradients together."""
    N, M = 11, 32
    phi = inputs.random_phases(41, 1, N)[0].astype(np.float64)
    s = orc.signal_from_phase(phi)
    gs, gphi, _ = orc.grad(s, M, orc.full_window(N, M), 1.0, 1.0, 50.0, 1e-12)
    np.testing.assert_allclose(np.real(np.conj(gs) * 1j * s), gphi, rtol=1e-12, atol=1e-14)
