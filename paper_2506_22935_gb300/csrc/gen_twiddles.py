"""Writes ``twiddles.inc`` for the CUDA library (run by the package build).

Two kinds of DFT twiddle factors W_L^q = exp(-2 pi j q / L) (the kernel of
Eq. 11 in the paper, M-point, negative exponent), each evaluated in float64 from
an exact integer ratio and rounded once to float32:

* ``graf_w64_re/im(q)``: constexpr switch functions for W_64^q, q in [0, 64).
  Every in-register radix-R butterfly (R | 64) uses W_R^q = W_64^(q * 64/R)
  with compile-time q, so these fold to immediates.
* ``g_tw_M<M>_p<p>``: per row length M and Stockham pass p >= 1 (radix R_p,
  span Ns_p = R_0 ... R_{p-1}), a table laid out [r-1][i] holding
  W_(Ns_p R_p)^(i r) for r in [1, R_p), i in [0, Ns_p).  Consecutive threads
  read consecutive i, so the loads coalesce.

The radix plan must match ``graf_fft.cuh``: R_0 = the values per thread
(32 from M = 512 on, 16 for M = 128 and 256, else min(M, 64)) and the rest
of M / R_0 is one pass if it is <= R_0, else 16 x (M / (16 R_0)).
"""
from __future__ import annotations

import math
import sys

M_ALL = [8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384]


def radix_plan(M: int) -> list[int]:
    r0 = 32 if M >= 512 else (16 if M >= 128 else min(M, 64))
    rest = M // r0
    if rest == 1:
        return [r0]
    if rest <= r0:
        return [r0, rest]
    return [r0, 16, rest // 16]


def w(q: int, L: int) -> tuple[float, float]:
    q %= L
    a = 2.0 * math.pi * q / L
    return math.cos(a), -math.sin(a)


def f32(x: float) -> str:
    import struct
    v = struct.unpack("f", struct.pack("f", x))[0]
    if v == 0.0:
        return "0.0f"
    s = f"{v:.9g}"
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


def main(out_path: str) -> None:
    lines = ["// generated by gen_twiddles.py: DFT twiddles exp(-2 pi j q / L), float64 -> float32",
             "#pragma once", ""]
    for part, idx in (("re", 0), ("im", 1)):
        lines.append(f"__host__ __device__ constexpr float graf_w64_{part}(int q) {{")
        lines.append("  switch (q & 63) {")
        for q in range(64):
            lines.append(f"    case {q}: return {f32(w(q, 64)[idx])};")
        lines.append("  }")
        lines.append("  return 0.0f;")
        lines.append("}")
    lines.append("")
    lines.append("template <int M, int P> struct GrafTw;")
    for M in M_ALL:
        plan = radix_plan(M)
        ns = plan[0]
        for p in range(1, len(plan)):
            R = plan[p]
            L = ns * R
            vals = []
            for r in range(1, R):
                for i in range(ns):
                    c, s = w(i * r, L)
                    vals.append(f"{{{f32(c)},{f32(s)}}}")
            lines.append(f"__device__ const float2 g_tw_M{M}_p{p}[{len(vals)}] = {{")
            for k in range(0, len(vals), 8):
                lines.append("  " + ",".join(vals[k:k + 8]) + ",")
            lines.append("};")
            lines.append(f"template <> struct GrafTw<{M}, {p}> {{ static __device__ __forceinline__ "
                         f"const float2* get() {{ return g_tw_M{M}_p{p}; }} }};")
            ns = L
        lines.append("")
    with open(out_path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1])
