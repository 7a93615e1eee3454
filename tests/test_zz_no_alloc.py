"""graf_af_loss_backward_noalloc: the entry point for callers that cannot
allocate device memory (fixed memory maps, host pools that own all device
memory, no tolerance for cudaMalloc's synchronisation).  It must give the
same loss scalars and gradient as graf_af_loss_backward with a caller
workspace, on consecutive calls that reuse its fixed scratch array.

This file is collected last on purpose, so a stop-at-first-failure run has
already run every other test if this one fails."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2506_22935_gb300 import _build, inputs
from paper_2506_22935_gb300 import graf as g

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G_TOL = 1e-4
L_TOL = 1e-5


def _with_workspace(x, kind, B, N, M, w, loss, grad_s, grad_phi):
    nb = g.graf_af_backward_workspace_bytes(B, N, M, w.c())
    ws = torch.empty(nb, dtype=torch.uint8, device=x.device)
    out8 = torch.empty((B, 8), dtype=torch.float32, device=x.device)
    st = g.graf_af_loss_backward(x.data_ptr(), kind, B, N, M, w.c(), loss.c(), out8.data_ptr(), None,
                                 None if grad_s is None else grad_s.data_ptr(),
                                 None if grad_phi is None else grad_phi.data_ptr(), ws.data_ptr(), nb,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == 0, g.graf_status_string(st)
    return out8


def _no_alloc(x, kind, B, N, M, w, loss, grad_s, grad_phi):
    out8 = torch.empty((B, 8), dtype=torch.float32, device=x.device)
    st = g.graf_af_loss_backward_noalloc(x.data_ptr(), kind, B, N, M, w.c(), loss.c(), out8.data_ptr(), None,
                                         None if grad_s is None else grad_s.data_ptr(),
                                         None if grad_phi is None else grad_phi.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert st == 0, g.graf_status_string(st)
    return out8


def _rel(a, b):
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def test_no_alloc_matches_workspace_path_on_consecutive_calls():
    _build.build()
    g.load()
    dev = torch.device("cuda:0")
    cases = [
        # two calls in a row on the shared scratch: the headline batch shape,
        # then a different shape and input kind
        ("phase", 256, 1024, 2048, g.Window.full(1024, 2048), g.Loss(1.0, 1.0, 50.0, 1e-12)),
        ("complex", 7, 300, 1024, g.Window(-40, 35, -200, 150, 0, 0), g.Loss(0.5, 1.0, 20.0, 1e-12)),
        ("phase", 256, 1024, 2048, g.Window.full(1024, 2048), g.Loss(1.0, 1.0, 50.0, 1e-12)),
    ]
    for i, (kind, B, N, M, w, loss) in enumerate(cases):
        if kind == "phase":
            x = torch.from_numpy(inputs.random_phases(500 + i, B, N)).to(dev)
            ga, gb = (torch.empty((B, N), dtype=torch.float32, device=dev) for _ in range(2))
            ref8 = _with_workspace(x, g.GRAF_IN_PHASE, B, N, M, w, loss, None, ga)
            got8 = _no_alloc(x, g.GRAF_IN_PHASE, B, N, M, w, loss, None, gb)
        else:
            x = torch.from_numpy(inputs.random_complex(500 + i, B, N)).to(dev)
            ga, gb = (torch.empty((B, N), dtype=torch.complex64, device=dev) for _ in range(2))
            ref8 = _with_workspace(x, g.GRAF_IN_COMPLEX, B, N, M, w, loss, ga, None)
            got8 = _no_alloc(x, g.GRAF_IN_COMPLEX, B, N, M, w, loss, gb, None)
        torch.cuda.synchronize()
        assert torch.allclose(got8, ref8, rtol=L_TOL, atol=0.0)
        for b in range(B):
            assert _rel(gb[b], ga[b]) <= G_TOL


def test_no_alloc_rejects_shapes_beyond_its_scratch():
    g.load()
    w = g.Window.full(8192, 16384)
    need = g.graf_af_backward_workspace_bytes(4096, 8192, 16384, w.c())
    assert need > (64 << 20)
    x = torch.zeros((1, 1), device="cuda:0")  # never read: the call is rejected first
    out8 = torch.empty((1, 8), device="cuda:0")
    st = g.graf_af_loss_backward_noalloc(x.data_ptr(), g.GRAF_IN_PHASE, 4096, 8192, 16384, w.c(), g.Loss().c(),
                                         out8.data_ptr(), None, None, out8.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert st == 7  # GRAF_ERR_WORKSPACE


def test_no_alloc_in_a_caller_created_context():
    """The scratch array's address is looked up in the context current at
    each call: calls in the primary context, in a context the caller creates
    with the driver API, and in the primary context again all match the
    workspace path (run in a child process that never loads torch)."""
    _build.build()
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "noalloc_context_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    rep = json.loads(r.stdout.strip().splitlines()[-1])
    assert rep["ok"], rep
