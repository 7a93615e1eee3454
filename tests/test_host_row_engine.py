"""Host-side checks of the CUDA row engine's compile-time parts, on the CPU:
the row plan of every length M against the twiddle generator's radix plan
(the two must agree or the per-pass tables index the wrong factors), the
generated twiddle factors against exp(-2 pi j q / L), and the in-register
R-point DFTs (R = 2..64, forward, inverse, zero-input and half-output forms)
against a direct double-precision DFT.  The host program is compiled by nvcc
as plain host code; nothing touches a GPU."""
import math
import os
import re
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_22935_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_twiddles  # noqa: E402


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def built(tmp_path_factory):
    d = tmp_path_factory.mktemp("row_engine")
    inc = d / "twiddles.inc"
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_twiddles.py"), str(inc)])
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = d / "row_engine_host"
    src = os.path.join(ROOT, "tests", "host", "row_engine_host.cu")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-I", CSRC, "-I", str(d),
                           "-x", "cu", src, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return out, inc.read_text()


def test_row_plan_matches_twiddle_generator(built):
    out, _ = built
    plans = [list(map(int, l.split()[1:])) for l in out.splitlines() if l.startswith("plan ")]
    assert [p[0] for p in plans] == gen_twiddles.M_ALL
    for M, vals, tpr, threads, npass, r0, r1, r2 in plans:
        radices = [r for r in (r0, r1, r2) if r > 1] or [1]
        assert radices == gen_twiddles.radix_plan(M), M
        assert len(gen_twiddles.radix_plan(M)) == npass
        assert math.prod(radices) == M and vals * tpr == M
        assert threads % tpr == 0 and threads <= 1024 and threads % 32 == 0


def test_register_dfts_match_direct_dft(built):
    out, _ = built
    errs = {int(l.split()[1]): float(l.split()[2]) for l in out.splitlines() if l.startswith("dft ")}
    assert sorted(errs) == [2, 4, 8, 16, 32, 64]
    for R, e in errs.items():
        # FP32 transform of inputs in [-1/2, 1/2]^2: about u log2(R) ||x||_2, ||x||_2 <= sqrt(R/2)
        assert e <= 4 * 2.0 ** -24 * math.log2(R) * math.sqrt(R / 2), (R, e)


def _floats(body):
    return [float(v.rstrip("f")) for v in re.findall(r"-?[0-9.]+(?:e[-+]?[0-9]+)?f", body)]


def test_generated_twiddles_are_the_dft_kernel(built):
    _, text = built
    # W_64^q = exp(-2 pi j q / 64) for the in-register butterflies
    for part, f in (("re", np.cos), ("im", lambda a: -np.sin(a))):
        body = re.search(r"graf_w64_%s\(int q\) \{(.*?)\n\}" % part, text, re.S).group(1)
        cases = {int(q): float(v.rstrip("f")) for q, v in re.findall(r"case (\d+): return ([^;]+);", body)}
        assert sorted(cases) == list(range(64))
        for q, v in cases.items():
            assert abs(v - f(2 * np.pi * q / 64)) <= 6e-8, (part, q)
    # per-pass tables [r-1][i] = W_(Ns R)^(i r)
    tables = re.findall(r"g_tw_M(\d+)_p(\d+)\[(\d+)\] = \{(.*?)\};", text, re.S)
    assert tables
    for M, p, n, body in tables:
        M, p, n = int(M), int(p), int(n)
        plan = gen_twiddles.radix_plan(M)
        ns, R = math.prod(plan[:p]), plan[p]
        v = np.array(_floats(body)).reshape(-1, 2)
        assert n == (R - 1) * ns == v.shape[0], (M, p)
        r = np.repeat(np.arange(1, R), ns)
        i = np.tile(np.arange(ns), R - 1)
        want = np.exp(-2j * np.pi * (i * r % (ns * R)) / (ns * R))
        assert np.abs(v[:, 0] + 1j * v[:, 1] - want).max() <= 1.2e-7, (M, p)
