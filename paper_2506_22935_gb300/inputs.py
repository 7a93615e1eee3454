"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the bench.  This module holds no arithmetic of the method itself: it only
draws numbers.

Generator: splitmix64 (S. Vigna's published 64-bit mixer), output i of a
stream with seed S is mix(S + (i+1) * 0x9E3779B97F4A7C15); a uniform double
is u = (x >> 11) * 2^-53.  Phases are phi = 2*pi*u rounded to float32, the
random polyphase codes of the paper's experiments (Sec. 7.1.2: phase-coded,
constant-modulus waveforms).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2506229350
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` consecutive splitmix64 outputs (uint64) starting at ``offset``."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): (x >> 11) * 2^-53."""
    x = splitmix64(seed, count, offset)
    return (x >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_phases(seed: int, batch: int, n: int) -> np.ndarray:
    """float32 [batch, n] i.i.d. uniform on [0, 2 pi)."""
    u = uniform(seed, batch * n).reshape(batch, n)
    return (2.0 * math.pi * u).astype(np.float32)


def lfm_phases(n: int) -> np.ndarray:
    """Discrete LFM chirp phi[k] = pi k^2 / n (time-bandwidth n), float32."""
    k = np.arange(n, dtype=np.float64)
    return (math.pi * k * k / n).astype(np.float32)


def random_complex(seed: int, batch: int, n: int) -> np.ndarray:
    """complex64 [batch, n] with independent uniform(-1, 1) real and imaginary
    parts: general (non unit-modulus) signals for the complex-input path."""
    u = uniform(seed, 2 * batch * n).reshape(batch, n, 2) * 2.0 - 1.0
    return (u[..., 0] + 1j * u[..., 1]).astype(np.complex64)


def uneven_lengths(seed: int, count: int, n_min: int = 128, n_max: int = 8192) -> np.ndarray:
    """int32 lengths log-uniform on [n_min, n_max]: round(exp(U[ln n_min, ln n_max]))."""
    u = uniform(seed, count)
    a, b = math.log(n_min), math.log(n_max)
    n = np.rint(np.exp(a + (b - a) * u)).astype(np.int64)
    return np.clip(n, n_min, n_max).astype(np.int32)


def barker13() -> np.ndarray:
    """The length-13 Barker code (+1 x5, -1 x2, +1 x2, -1, +1, -1, +1), a
    textbook binary sequence whose aperiodic autocorrelation sidelobes are at
    most 1 in magnitude."""
    return np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1], dtype=np.float64)
