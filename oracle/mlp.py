"""FP64 reference of the learned proposal MLP and its phase label loss (test
infrastructure; only tests, smoke and the bench's reference legs use it).

spec[8] -> W1 (16 x 512, inputs zero-padded to 16) -> GELU -> W2 (512 x 512)
-> GELU -> W3 (512 x 1024) -> phases.  With ``bf16=True`` every value the
CUDA path stores in BF16 is rounded to BF16 (round to nearest even) at the
same point: the padded input, the weights, the hidden activations and the
backward's output gradient and pre-activation gradients; all arithmetic is
float64 otherwise.  GELU(x) = x Phi(x) with the exact normal CDF.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

IN, IN_PAD, HID, OUT = 8, 16, 512, 1024
SHAPES = [("W1", (IN_PAD, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, OUT)), ("b3", (OUT,))]


def param_count() -> int:
    return sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(spec, flat, bf16_round=True):
    """Returns (phases, cache)."""
    r = bf16 if bf16_round else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(flat)
    spec = np.asarray(spec, dtype=np.float64)
    x16 = np.zeros((spec.shape[0], IN_PAD))
    x16[:, :IN] = spec
    x16 = r(x16)
    pre1 = x16 @ r(p["W1"]) + p["b1"]
    h1 = r(gelu(pre1))
    pre2 = h1 @ r(p["W2"]) + p["b2"]
    h2 = r(gelu(pre2))
    out = h2 @ r(p["W3"]) + p["b3"]
    return out, dict(x16=x16, pre1=pre1, h1=h1, pre2=pre2, h2=h2, r=r, p=p)


def label_loss(pred, target, scale=1.0):
    """Per row min over s = +-1 of 1 - |mean_n exp(j (pred - s target))| and
    scale * dL/dpred (a global phase and conjugation of the target leave it
    unchanged).  Returns (loss[rows], grad[rows, n])."""
    pred = np.asarray(pred, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    n = pred.shape[1]
    loss = np.empty(pred.shape[0])
    grad = np.empty_like(pred)
    for b in range(pred.shape[0]):
        best = None
        for s in (1.0, -1.0):
            th = pred[b] - s * target[b]
            z = np.mean(np.exp(1j * th))
            if best is None or abs(z) > abs(best[0]):
                best = (z, th)
        z, th = best
        loss[b] = 1.0 - abs(z)
        grad[b] = scale * np.imag(np.conj(z) * np.exp(1j * th)) / (n * abs(z)) if abs(z) > 0 else 0.0
    return loss, grad


def backward(cache, dout):
    """Gradient (flat, parameter layout) of sum(dout * phases)."""
    r, p = cache["r"], cache["p"]
    dy3 = r(dout)
    g = {}
    g["W3"] = cache["h2"].T @ dy3
    g["b3"] = dy3.sum(axis=0)
    dpre2 = r((dy3 @ r(p["W3"]).T) * gelu_grad(cache["pre2"]))
    g["W2"] = cache["h1"].T @ dpre2
    g["b2"] = dpre2.sum(axis=0)
    dpre1 = r((dpre2 @ r(p["W2"]).T) * gelu_grad(cache["pre1"]))
    g["W1"] = cache["x16"].T @ dpre1
    g["b1"] = dpre1.sum(axis=0)
    return pack(g)
