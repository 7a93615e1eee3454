"""The cuFFT comparison pipeline of the bench (eager torch + torch.fft, run
here on the CPU) computes the same loss and phase gradient as the oracle:
a timed comparison is only meaningful if it does the same work."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
import oracle
from paper_2506_22935_gb300 import inputs


@pytest.mark.parametrize("Ns,M", [([16, 11, 5], 32), ([24, 24], 64), ([100, 64], 256)])
def test_cufft_pipeline_matches_oracle(Ns, M):
    nmax = max(Ns)
    phi = np.zeros((len(Ns), nmax), dtype=np.float32)
    raw = inputs.random_phases(77, len(Ns), nmax)
    for b, n in enumerate(Ns):
        phi[b, :n] = raw[b, :n]
    box = np.array([max(M // n - 1, 0) for n in Ns])
    L, gphi = bench.cufft_loss_grad(torch.from_numpy(phi).double().float(), torch.tensor(Ns), M,
                                    torch.from_numpy(box), 50.0, 1e-12, chunk=2)
    for b, n in enumerate(Ns):
        s = oracle.signal_from_phase(phi[b, :n].astype(np.float64))
        win = (-(n - 1), n - 1, -(M // 2), M // 2 - 1, 0, int(box[b]))
        _, gp, out = oracle.grad(s, M, win, 1.0, 1.0, 50.0, 1e-12)
        assert abs(float(L[b]) - out[0]) <= 1e-5 * abs(out[0])
        g = gphi[b, :n].double().numpy()
        assert np.linalg.norm(g - gp) <= 1e-4 * np.linalg.norm(gp) + 1e-7
        assert np.all(gphi[b, n:].numpy() == 0)
