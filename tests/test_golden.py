"""Published values (fixtures under tests/golden/, each citing its source)
against the FP64 oracle and, on a GPU, against the CUDA path."""
import os

import numpy as np
import pytest

import oracle as orc
from paper_2506_22935_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _barker_acf():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "barker13_acf.txt")) if ln.strip() and ln[0] != "#"]
    acf = np.array([float(r[1]) for r in rows])
    assert [int(r[0]) for r in rows] == list(range(13))
    return acf


@pytest.mark.parametrize("M", [32, 64])
def test_oracle_zero_doppler_row_is_the_published_barker13_autocorrelation(M):
    """X[k, 0] of the oracle (Eq. 8 and Eq. 11 at m = 0) for k = -12 .. 12
    equals the tabulated autocorrelation, exactly (integer arithmetic in FP64)."""
    acf = _barker_acf()
    s = inputs.barker13().astype(np.complex128)
    X = orc.af_complex(s, M, -12, 12, 0, 0)[:, 0]
    want = np.concatenate([acf[:0:-1], acf])  # k = -12 .. 12
    np.testing.assert_array_equal(X.real, want)
    np.testing.assert_array_equal(X.imag, np.zeros(25))


@pytest.mark.gpu
def test_gpu_zero_doppler_row_is_the_published_barker13_autocorrelation():
    """The CUDA forward (complex input) returns Ahat = sqrt(|X|^2 + eps) / E
    with E = 13; at m = 0, E * Ahat is |R[k]| of the table within FP32
    rounding."""
    torch = pytest.importorskip("torch")
    from paper_2506_22935_gb300 import _build
    from paper_2506_22935_gb300 import graf as g
    _build.build()
    g.load()
    acf = _barker_acf()
    N, M = 13, 32
    s = torch.from_numpy(inputs.barker13().astype(np.complex64)[None, :]).to("cuda:0")
    w = g.Window(-12, 12, 0, 0, 0, 0)
    A = g.af_forward(s, M, w, 0.0).cpu().numpy()[0][:, 0]
    want = np.concatenate([acf[:0:-1], acf]) / 13.0
    assert np.abs(A - want).max() <= 1e-6
