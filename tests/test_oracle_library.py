"""Pins of the AF oracles against a library routine on general inputs: every
delay row of the AF is the DFT of that row's lag product (Eq. 8, Eq. 11;
Eq. 7 for the periodic form), so numpy's FFT of the lag product, built here
from the definition, must reproduce the oracles' direct double sums cell by
cell.  The oracles use no FFT, so an index, sign or conjugation slip in their
sums fails here.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2506_22935_gb300 import inputs


def _lag(s, k):
    """R[k,n] = s[n] conj(s[n-k]) for n in [0, N), zero where n-k is outside."""
    N = s.shape[0]
    R = np.zeros(N, dtype=np.complex128)
    for n in range(N):
        if 0 <= n - k < N:
            R[n] = s[n] * np.conj(s[n - k])
    return R


@pytest.mark.parametrize("N,M", [(5, 8), (13, 16), (16, 16), (24, 64), (31, 32)])
def test_aperiodic_rows_are_ffts_of_lag_products(N, M):
    s = inputs.random_complex(90 + N, 1, N)[0].astype(np.complex128)
    X = oracle.af_complex(s, M, -(N - 1), N - 1, -(M // 2), M // 2 - 1, nthreads=1)
    for i, k in enumerate(range(-(N - 1), N)):
        R = np.zeros(M, dtype=np.complex128)
        R[:N] = _lag(s, k)
        F = np.fft.fft(R)                      # sum_n R[n] exp(-2 pi j m n / M)
        want = np.fft.fftshift(F)              # m = -M/2 .. M/2-1
        np.testing.assert_allclose(X[i], want, rtol=0, atol=1e-12 * N * N)


@pytest.mark.parametrize("N", [8, 16, 32])
@pytest.mark.parametrize("sign", [1, -1])
def test_periodic_rows_are_ffts_of_circular_lag_products(N, sign):
    s = inputs.random_complex(95 + N, 1, N)[0].astype(np.complex128)
    X = oracle.paf_complex(s, sign)
    for i, k in enumerate(range(-(N // 2), N - N // 2)):
        R = s * np.conj(np.roll(s, k))         # s[n] conj(s[(n-k) mod N])
        F = np.fft.fft(R) if sign < 0 else np.fft.ifft(R) * N
        np.testing.assert_allclose(X[i], np.fft.fftshift(F), rtol=0, atol=1e-12 * N * N)
