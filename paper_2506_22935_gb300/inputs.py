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


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal draws (Box-Muller on pairs of uniforms)."""
    m = (count + 1) // 2
    u1 = uniform(seed, m, 2 * offset)
    u2 = uniform(seed, m, 2 * offset + m)
    r = np.sqrt(-2.0 * np.log(1.0 - u1))
    z = np.concatenate([r * np.cos(2 * math.pi * u2), r * np.sin(2 * math.pi * u2)])
    return z[:count]


def design_specs(seed: int, count: int) -> dict:
    """Design specs of the learned proposal: delay-mask half-width K log-uniform
    on [16, 512], Doppler-mask half-width Mw log-uniform on [8, 256] (both
    rounded), PSL and ISL weights uniform on [0, 1] (ISL weight at least 0.1),
    and four standard-normal noise dimensions."""
    u = uniform(seed, 4 * count).reshape(count, 4)
    K = np.rint(np.exp(math.log(16) + u[:, 0] * (math.log(512) - math.log(16)))).astype(np.int32)
    Mw = np.rint(np.exp(math.log(8) + u[:, 1] * (math.log(256) - math.log(8)))).astype(np.int32)
    w_psl = u[:, 2]
    w_isl = 0.1 + 0.9 * u[:, 3]
    noise = normal(seed + 1, 4 * count).reshape(count, 4)
    return dict(K=K, Mw=Mw, w_psl=w_psl, w_isl=w_isl, noise=noise)


def spec_features(specs: dict) -> np.ndarray:
    """float32 [count, 8]: log-widths mapped to [-1, 1], the two weights, the
    noise dimensions."""
    k = (np.log(specs["K"]) - math.log(16)) / (math.log(512) - math.log(16)) * 2.0 - 1.0
    m = (np.log(specs["Mw"]) - math.log(8)) / (math.log(256) - math.log(8)) * 2.0 - 1.0
    f = np.concatenate([k[:, None], m[:, None], specs["w_psl"][:, None], specs["w_isl"][:, None],
                        specs["noise"]], axis=1)
    return f.astype(np.float32)


def mlp_init_params(seed: int) -> np.ndarray:
    """float64 flat parameters of the 8(16)->512->512->1024 MLP: weights
    uniform(-a, a) with a = sqrt(6 / (fan_in + fan_out)) (Glorot), zero rows
    for the input padding, zero biases.  Layout W1 [16][512] | b1 | W2
    [512][512] | b2 | W3 [512][1024] | b3."""
    shapes = [("W", 16, 512, 8), ("b", 512), ("W", 512, 512, 512), ("b", 512), ("W", 512, 1024, 512),
              ("b", 1024)]
    parts, off = [], 0
    for s in shapes:
        if s[0] == "W":
            _, rows, cols, fan_in = s
            n = rows * cols
            a = math.sqrt(6.0 / (fan_in + cols))
            w = ((uniform(seed, n, off) * 2.0 - 1.0) * a).reshape(rows, cols)
            w[fan_in:, :] = 0.0
            parts.append(w.ravel())
        else:
            n = s[1]
            parts.append(np.zeros(n))
        off += n
    return np.concatenate(parts)
