"""Child process of tests/test_zz_no_alloc.py (not collected by pytest).

Runs graf_af_loss_backward_noalloc in two CUDA contexts of one device: the
primary context, then a context this process creates itself with the driver
API (which the CUDA runtime inside the library then uses), then the primary
context again.  The library's fixed scratch array has a different device
address in each context, so a call that reused an address from an earlier
context would address memory of another context.  Each call's loss scalars
and gradient are compared with graf_af_loss_backward given a workspace
allocated in the primary context.  Device memory comes from the driver API
(cuMemAlloc), so torch is not loaded.  Prints one JSON line; exit code 0
when every comparison passes.
"""
import ctypes
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2506_22935_gb300 import graf as g  # noqa: E402
from paper_2506_22935_gb300 import inputs  # noqa: E402

B, N, M = 3, 200, 512
G_TOL, L_TOL = 1e-4, 1e-5


def main():
    cu = ctypes.CDLL("libcuda.so.1")
    u64 = ctypes.c_uint64

    def ck(r, what):
        if r != 0:
            raise RuntimeError(f"{what} failed with CUresult {r}")

    ck(cu.cuInit(0), "cuInit")
    dev = ctypes.c_int()
    ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
    primary = ctypes.c_void_p()
    ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(primary), dev), "cuDevicePrimaryCtxRetain")
    ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")

    lib = g.load()
    w, loss = g.Window.full(N, M), g.Loss(1.0, 1.0, 50.0, 1e-12)
    phi = np.ascontiguousarray(inputs.random_phases(inputs.SEED_BASE + 900, B, N))

    def alloc(nbytes):
        p = u64()
        ck(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nbytes)), "cuMemAlloc")
        return p.value

    def run(noalloc):
        """One call in the current context; returns (out8, grad) on the host."""
        x = alloc(phi.nbytes)
        o8 = alloc(B * 8 * 4)
        gd = alloc(B * N * 4)
        ck(cu.cuMemcpyHtoD_v2(u64(x), phi.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(phi.nbytes)), "HtoD")
        if noalloc:
            st = lib.graf_af_loss_backward_noalloc(x, g.GRAF_IN_PHASE, B, N, M, w.c(), loss.c(), o8, None, None,
                                                   gd, None)
        else:
            nb = g.graf_af_backward_workspace_bytes(B, N, M, w.c())
            ws = alloc(nb)
            st = lib.graf_af_loss_backward(x, g.GRAF_IN_PHASE, B, N, M, w.c(), loss.c(), o8, None, None, gd, ws,
                                           nb, None)
        if st != 0:
            raise RuntimeError(f"graf call failed: {g.graf_status_string(st)}")
        ck(cu.cuCtxSynchronize(), "cuCtxSynchronize")
        out8 = np.empty((B, 8), dtype=np.float32)
        grad = np.empty((B, N), dtype=np.float32)
        ck(cu.cuMemcpyDtoH_v2(out8.ctypes.data_as(ctypes.c_void_p), u64(o8), ctypes.c_size_t(out8.nbytes)), "DtoH")
        ck(cu.cuMemcpyDtoH_v2(grad.ctypes.data_as(ctypes.c_void_p), u64(gd), ctypes.c_size_t(grad.nbytes)), "DtoH")
        return out8, grad

    ref8, refg = run(noalloc=False)
    results = {"primary": run(noalloc=True)}
    created = ctypes.c_void_p()
    # a context of this process's own making (cuCtxCreate_v4 with no
    # parameters); it becomes current, and the runtime uses it
    ck(cu.cuCtxCreate_v4(ctypes.byref(created), None, 0, dev), "cuCtxCreate")
    results["created"] = run(noalloc=True)
    ck(cu.cuCtxSetCurrent(primary), "cuCtxSetCurrent")
    results["primary_again"] = run(noalloc=True)

    report, ok = {}, True
    for name, (o8, gd) in results.items():
        lrel = float(np.max(np.abs(o8 - ref8) / np.maximum(np.abs(ref8), 1e-30)))
        grel = max(float(np.linalg.norm(gd[b] - refg[b]) / np.linalg.norm(refg[b])) for b in range(B))
        report[name] = {"loss_max_rel": lrel, "grad_max_rel_l2": grel}
        ok &= lrel <= L_TOL and grel <= G_TOL
    ck(cu.cuCtxDestroy_v2(created), "cuCtxDestroy")
    print(json.dumps({"ok": bool(ok), **report}), flush=True)
    return 0 if ok else 1


if __name__ == "__main__":
    sys.exit(main())
