"""Pins for the target-matching reference (L_match of Eq. 22): a target equal
to the code's own surface, a zero target against the AF oracle's cells, and
finite differences.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2506_22935_gb300 import inputs


def _ahat2(s, M, w, eps=1e-12):
    return oracle.af_ahat(s, M, w[0], w[1], w[2], w[3], eps) ** 2


@pytest.mark.parametrize("w", [(-7, 7, -8, 7, 0, 0), (-3, 5, -2, 6, -1, -1)])
def test_own_surface_and_zero_target(w):
    N, M = 8, 16
    s = inputs.random_complex(3, 1, N)[0].astype(np.complex128)
    own = _ahat2(s, M, w)
    loss, gs, _ = oracle.match(s, M, w, own, 1.0)
    assert loss < 1e-24 and np.abs(gs).max() < 1e-10
    loss0, _, _ = oracle.match(s, M, w, np.zeros_like(own), 1.0)
    assert abs(loss0 - np.sum(own ** 2)) < 1e-12 * np.sum(own ** 2)


def test_match_gradient_matches_finite_differences():
    N, M = 10, 32
    w = (-9, 9, -16, 15, -1, -1)
    rng = np.random.default_rng(4)
    target = rng.random((19, 32)) * 0.05
    z = inputs.random_complex(5, 1, N)[0].astype(np.complex128)
    _, gz, _ = oracle.match(z, M, w, target, 0.7)
    h = 1e-6
    fd = np.zeros(N, dtype=np.complex128)
    for i in range(N):
        for unit in (1.0, 1j):
            a, b = z.copy(), z.copy()
            a[i] += h * unit
            b[i] -= h * unit
            fd[i] += unit * 0.7 * (oracle.match(a, M, w, target)[0] - oracle.match(b, M, w, target)[0]) / (2 * h)
    assert np.linalg.norm(gz - fd) <= 1e-6 * np.linalg.norm(fd)
    phi = inputs.random_phases(6, 1, N)[0].astype(np.float64)
    _, _, gp = oracle.match(np.exp(1j * phi), M, w, target, 0.7)
    fdp = np.zeros(N)
    for i in range(N):
        a, b = phi.copy(), phi.copy()
        a[i] += h
        b[i] -= h
        fdp[i] = 0.7 * (oracle.match(np.exp(1j * a), M, w, target)[0] -
                        oracle.match(np.exp(1j * b), M, w, target)[0]) / (2 * h)
    assert np.linalg.norm(gp - fdp) <= 1e-6 * np.linalg.norm(fdp)
