"""Benchmark: batched ambiguity-function forward + backward on GB300.

Workload: 256 random polyphase codes (phases i.i.d. uniform on [0, 2 pi),
seeded), N = 1024, M = 2048, all 2047 delays and 2048 Doppler bins, loss
PSL_soft (log-sum-exp, beta = 50) + ISL over the AF minus the zero-delay
mainlobe, forward and Wirtinger backward with respect to the phases, FP32.
One step = graf_af_loss_backward over the batch (fused loss + gradient);
metric = AF cells per second, cells = B (2N-1) M per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun, one rank per GPU, each on its own batch (weak
scaling, no data-path collective).  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

B, N, M = 256, 1024, 2048
BETA, EPS = 50.0, 1e-12
SEED = 2506229350 + 2
METRIC = "AF fwd+bwd Gcells/s at N=1024 M=2048"
UNIT = "Gcells/s"
WORKLOAD = ("256 random polyphase codes, N=1024, M=2048, all 2047 delays x 2048 Doppler bins, "
            "PSL(log-sum-exp beta=50)+ISL, forward + Wirtinger backward w.r.t. phases")
FLOP_PER_ROW = 5.0 * M * math.log2(M)  # nominal radix-2 count of one M-point FFT
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell: 4 partitions x 32)


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def rank_seed(rank: int) -> int:
    """Each rank draws its own batch (weak scaling: independent waveforms)."""
    return SEED + 1000 * rank


def reduce_max_ms(ms: float, dist, device) -> float:
    """The slowest rank's time (the job's time); a no-op without a process group."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world: int, cells_per_rank: float, steps: int, total_ms: float) -> float:
    """Whole-job Gcells/s: every rank's cells over the slowest rank's time."""
    return world * cells_per_rank * steps / (total_ms / 1e3) / 1e9


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _fp32_peak(dev):
    """FP32 FMA peak of `dev` in TFLOP/s: the SM count read from the device
    (cudaDevAttrMultiProcessorCount through torch) x 128 lanes x 2 flop x the
    maximum SM clock of MEASURED_PEAKS.json; and how it was formed."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, src = _measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sms * FP32_LANES * 2 * mhz * 1e6 / 1e12
    return peak, (f"FP32 FMA peak = {sms} SMs (read from the device) x {FP32_LANES} lanes x 2 x {mhz:.0f} MHz "
                  f"(sm_max_mhz from MEASURED_PEAKS.json, {src})")


# the sources af_fused_kernel<2048> is compiled from
_FUSED_SOURCES = ("graf_af_impl.cuh", "graf_fft.cuh", "graf_kernels.cuh", "graf_af_m2048.cu", "gen_twiddles.py")


def _kernel_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2506_22935_gb300", "csrc")
    for name in _FUSED_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def _traffic_record():
    """DRAM bytes per launch of the fused kernel (from an ncu capture of a
    32-code slice, scaled to the full batch), valid only if the kernel sources
    are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f)
    if rec.get("source_hash") != _kernel_hash():
        return None
    return rec.get("af_fused_bytes_per_launch_full_batch")


class ClockSampler:
    """SM clock, power and clock-event reasons sampled in-process through
    NVML (read-only queries, libnvidia-ml via ctypes) every `period` seconds
    on a background thread while the `with` block runs.  Samples whose
    reasons include "GPU idle" are not counted as under load."""
    # NVML clock-event reason bits (nvml.h: nvmlClocksEventReason*)
    IDLE, SW_POWER_CAP, HW_SLOWDOWN, SW_THERMAL, HW_THERMAL, HW_POWER_BRAKE = 0x1, 0x4, 0x8, 0x20, 0x40, 0x80
    NAMES = ((SW_POWER_CAP, "sw_power_cap"), (HW_SLOWDOWN, "hw_slowdown"), (SW_THERMAL, "sw_thermal_slowdown"),
             (HW_THERMAL, "hw_thermal_slowdown"), (HW_POWER_BRAKE, "hw_power_brake_slowdown"))

    def __init__(self, device, period: float = 0.01):
        self.device, self.period = device, period
        self.samples, self.error = [], None
        self._stop = None
        self._thread = None
        self._nvml = self._handle = None

    def _open(self):
        import ctypes
        import torch
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit_v2 failed")
        h = ctypes.c_void_p()
        uuid = getattr(torch.cuda.get_device_properties(self.device), "uuid", None)
        ok = False
        if uuid is not None:
            u = str(uuid)
            u = u if u.startswith("GPU-") else "GPU-" + u
            ok = nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
        if not ok:
            idx = self.device.index if self.device.index is not None else 0
            if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) != 0:
                raise OSError("no NVML handle for the device")
        self._nvml, self._handle = nv, h
        reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self._reasons = reasons if reasons is not None else nv.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))  # NVML_CLOCK_SM = 1
        self.max_mhz = float(mx.value)

    def _run(self):
        import ctypes
        nv, h = self._nvml, self._handle
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                    self._reasons(h, ctypes.byref(rs)) == 0:
                p = float(pw.value) / 1e3 if nv.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw)) == 0 else None
                self.samples.append((float(clk.value), int(rs.value), p))
            self._stop.wait(self.period)

    def __enter__(self):
        import threading
        try:
            self._open()
        except Exception as e:  # no NVML on this host: the line says so
            self.error = f"{type(e).__name__}: {e}"
            return self
        self._stop = threading.Event()
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def __exit__(self, *a):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)

    def summary(self):
        if self.error is not None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples_under_load": 0,
                    "source": "NVML unavailable: " + self.error}
        load = [x for x in self.samples if not (x[1] & self.IDLE)]
        reasons = sorted({nm for _, r, _ in load for bit, nm in self.NAMES if r & bit})
        pw = [p for _, _, p in load if p is not None]
        return {"sm_mhz": statistics.median([c for c, _, _ in load]) if load else None,
                "sm_max_mhz": self.max_mhz, "reasons": reasons, "samples_under_load": len(load),
                "samples": len(self.samples), "power_w_max": max(pw) if pw else None,
                "source": f"NVML in-process, every {self.period * 1e3:.0f} ms across warm-up and timed steps"}


def _oracle_cols(cols, nthreads=None, want_grad=False):
    """FP64 oracle loss + gradient (forward + backward) of ONE waveform of the
    workload (waveform 0 of rank 0's batch) over all 2047 delays and `cols`
    Doppler bins centred on m = 0 (cols = M is the whole AF).  Every cell
    costs the same O(N - |k|) in the forward and O(1) per (k, n) in the
    adjoint, so a Doppler slice is a representative sample.  Returns (cells,
    seconds, cores) and, with want_grad, the phase gradient as well."""
    import numpy as np

    import oracle
    from paper_2506_22935_gb300 import inputs
    phi = inputs.random_phases(SEED, 1, N)[0].astype(np.float64)
    s = oracle.signal_from_phase(phi)
    m_lo = -(cols // 2)
    win = (-(N - 1), N - 1, m_lo, m_lo + cols - 1, 0, max(M // N - 1, 0))
    cores = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    _, gp, _ = oracle.grad(s, M, win, 1.0, 1.0, BETA, EPS, nthreads=cores)
    dt = time.perf_counter() - t0
    if want_grad:
        return (2 * N - 1) * cols, dt, cores, gp
    return (2 * N - 1) * cols, dt, cores


def _oracle_budget_cols(seconds):
    """Doppler bins of one waveform the oracle processes in about `seconds`."""
    _, dt, _ = _oracle_cols(8)
    cols = int(8 * seconds / max(dt, 1e-6))
    return max(1, min(M, cols))


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    budget = min(30.0, 150.0 / (args.steps + args.warmup))
    cols = _oracle_budget_cols(budget)
    for _ in range(args.warmup):
        _oracle_cols(cols)
    times, cells, cores = [], 0, 1
    for _ in range(args.steps):
        c, dt, cores = _oracle_cols(cols)
        times.append(dt)
        cells = c
    v = cells / statistics.mean(times) / 1e9
    sample = (f"per step: all 2047 delays x {cols} of {M} Doppler bins of 1 of {B} waveforms "
              f"(N={N}), FP64 loss + gradient")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (FP64 oracle, bounded sample per step)",
                                            "B": B, "N": N, "M": M},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_graf(args):
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    g.load()

    Bb = args.batch
    cells = Bb * (2 * N - 1) * M
    phi_h = inputs.random_phases(rank_seed(rank), Bb, N)
    x = torch.from_numpy(phi_h).to(dev)
    w, loss = g.Window.full(N, M), g.Loss(1.0, 1.0, BETA, EPS)
    wc, lc = w.c(), loss.c()
    nb = g.graf_af_backward_workspace_bytes(Bb, N, M, wc)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out8 = torch.empty((Bb, 8), dtype=torch.float32, device=dev)
    grad = torch.empty((Bb, N), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream

    def step_call(xp, o8p, gp):
        st = g.graf_af_loss_backward(xp, g.GRAF_IN_PHASE, Bb, N, M, wc, lc, o8p, None, None, gp, ws.data_ptr(),
                                     nb, sp)
        assert st == 0, g.graf_status_string(st)

    launches_per_step = 3  # fused rows, loss finalisation, gradient reduction
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    clk = ClockSampler(dev).__enter__()  # sampled through the timed and the end-to-end steps
    for _ in range(args.warmup):
        step_call(x.data_ptr(), out8.data_ptr(), grad.data_ptr())
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        e0, e1 = ev[i]
        e0.record(stream)
        step_call(x.data_ptr(), out8.data_ptr(), grad.data_ptr())
        e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms = reduce_max_ms(sum(e0.elapsed_time(e1) for e0, e1 in ev), dist, dev)
    ms_per_step = step_ms / args.steps
    value = weak_value(world, cells, args.steps, step_ms)
    assert torch.isfinite(out8).all() and torch.isfinite(grad).all()

    # end to end: pinned host phases in, loss scalars and gradient out, per step
    xh = torch.from_numpy(phi_h).pin_memory()
    o8h = torch.empty((Bb, 8), dtype=torch.float32).pin_memory()
    gh = torch.empty((Bb, N), dtype=torch.float32).pin_memory()
    xd = torch.empty_like(x)
    for _ in range(2):
        xd.copy_(xh, non_blocking=True)
        step_call(xd.data_ptr(), out8.data_ptr(), grad.data_ptr())
        o8h.copy_(out8, non_blocking=True)
        gh.copy_(grad, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xd.copy_(xh, non_blocking=True)
        step_call(xd.data_ptr(), out8.data_ptr(), grad.data_ptr())
        o8h.copy_(out8, non_blocking=True)
        gh.copy_(grad, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms += a.elapsed_time(b)
    clk.__exit__(None, None, None)
    e2e_value = weak_value(world, cells, args.steps, reduce_max_ms(e2e_ms, dist, dev))

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    cmp, cufft_g0 = None, None
    if world == 1 and not args.no_cufft:
        # the same step through cuFFT + eager torch ops (timed comparison only)
        nl = torch.full((Bb,), N, dtype=torch.int64, device=dev)
        fn = lambda: cufft_loss_grad(x, nl, M, max(M // N - 1, 0), BETA, EPS, chunk=32)
        ms_c, (lc_, gc_) = time_cufft(fn, 3, 1, stream)
        step_call(x.data_ptr(), out8.data_ptr(), grad.data_ptr())
        torch.cuda.synchronize(dev)
        cufft_g0 = gc_[0].double().cpu().numpy()
        cmp = {"value": cells / (ms_c / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms_c,
               "speedup_of_graf": ms_c / ms_per_step,
               "loss_max_rel_diff": float(((lc_ - out8[:, 0]).abs() / out8[:, 0].abs()).max()),
               "grad_rel_l2_diff": float((gc_ - grad).norm() / grad.norm()),
               "what": "torch.fft (cuFFT) row DFTs and inverse DFTs + eager torch lag products, magnitudes, "
                       "log-sum-exp and the hand-written adjoint with the kernels' exact split of the cell "
                       "adjoint (same loss and gradient), rows k >= 0 with mirror weights, 32 codes per chunk"}
        del lc_, gc_
        torch.cuda.empty_cache()

    fwd = run_forward_store(g, x, Bb, dev, stream, flush) if world == 1 and not args.no_forward_store else None
    learned_res = learned_eval(args, dev) if world == 1 and not args.no_learned else None

    peak_tflops, peak_src = _fp32_peak(dev)
    # algorithmic work of one call: the forward DFT and its adjoint for every
    # one of the 2N-1 delay rows; executed: both transforms for the N rows
    # k >= 0 (rows -k are mirrors), minus the adjoint of row 0
    alg = Bb * 2 * (2 * N - 1) * FLOP_PER_ROW
    executed = Bb * (2 * N - 1) * FLOP_PER_ROW
    achieved = alg / (ms_per_step / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": _traffic_record(),
                "kernel": "af_fused_kernel<2048> (+ loss finalisation and gradient reduction in the same timing)",
                "peak_source": peak_src,
                "algorithmic_flop_per_launch": alg,
                "executed_flop_per_launch": executed,
                "executed_frac": executed / (ms_per_step / 1e3) / 1e12 / peak_tflops}
    roofline["frac_basis"] = ("frac counts the algorithmic work, a forward DFT and its adjoint for every one "
                              "of the 2N-1 delay rows (the basis the >= 50% target is stated on); the kernel "
                              "executes half of it (rows k >= 0, |X[-k,m]| = |X[k,-m]|, and X reused by the "
                              "adjoint), so executed_frac is its use of the FP32 pipes")
    cpu, errors = None, None
    if world == 1 and not args.no_cpu_baseline:
        errors = fp64_errors(g, x, out8, grad, dev)
    if world == 1 and not args.no_cpu_baseline:
        import numpy as np
        cols = _oracle_budget_cols(15.0)
        cells, dt, cores, g_orc = _oracle_cols(cols, want_grad=True)
        cpu = {"value": cells / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"all 2047 delays x {cols} of {M} Doppler bins of 1 of {B} waveforms (N={N}), "
                         f"FP64 loss + gradient, {dt:.1f} s on {cores} threads"}
        if cols == M:
            # the whole AF of waveform 0: both GPU gradients against FP64
            rel = lambda a: float(np.linalg.norm(a - g_orc) / np.linalg.norm(g_orc))
            cpu["grad_rel_l2_graf_vs_oracle_wave0"] = rel(grad[0].double().cpu().numpy())
            errors["headline_B256_N1024_M2048"]["grad_rel_l2_wave0"] = rel(grad[0].double().cpu().numpy())
            if cufft_g0 is not None:
                cmp["grad_rel_l2_vs_oracle_wave0"] = rel(cufft_g0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if Bb == B else WORKLOAD.replace("256", str(Bb), 1),
                       "B_per_gpu": Bb, "N": N, "M": M, "beta": BETA, "eps": EPS,
                       "seed": SEED, "l2": "flushed between steps (256 MB write, outside the timed events)"},
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": Bb * N * 4,
                    "d2h_bytes_per_step": Bb * 8 * 4 + Bb * N * 4},
            "gpu_launches": launches_per_step * args.steps, "clocks": clk.summary(),
            "cufft_pipeline": cmp, "forward_store": fwd, "errors_vs_fp64": errors, "learned": learned_res}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_forward_store(g, x, Bb, dev, stream, flush, reps=5):
    """graf_af_forward over the whole AF of the benchmark batch (all 2N-1
    delays x M Doppler bins of every code: 4.29 GB of fp32 written at B =
    256), timed with CUDA events: Gcells/s, GB/s of output, its fraction of
    the measured HBM copy bandwidth, and the FP32 fraction of the forward
    DFTs (5 M log2 M flop per delay row; the kernel transforms rows k >= 0)."""
    import torch
    w = g.Window.full(N, M)
    out = torch.empty((Bb, 2 * N - 1, M), dtype=torch.float32, device=dev)
    sp = stream.cuda_stream

    def call():
        st = g.graf_af_forward(x.data_ptr(), g.GRAF_IN_PHASE, Bb, N, M, w.c(), EPS, out.data_ptr(), sp)
        assert st == 0, g.graf_status_string(st)

    ms = _timed_events(call, reps, 2, stream, flush)
    cells = Bb * (2 * N - 1) * M
    nbytes = 4.0 * cells
    peaks, src = _measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    peak_tf, _ = _fp32_peak(dev)
    alg = Bb * (2 * N - 1) * FLOP_PER_ROW
    exe = Bb * N * FLOP_PER_ROW
    gbs = nbytes / (ms / 1e3) / 1e9
    res = {"kernel": "af_forward_kernel<2048, N <= M/2>", "ms": ms, "Gcells_per_s": cells / (ms / 1e3) / 1e9,
           "bytes_written": nbytes, "GB_per_s": gbs, "hbm_frac": gbs / hbm,
           "hbm_peak_gbs": hbm, "hbm_peak_source": f"MEASURED_PEAKS.json hbm_gbs ({src})",
           "fp32_frac_algorithmic": alg / (ms / 1e3) / 1e12 / peak_tf,
           "fp32_frac_executed": exe / (ms / 1e3) / 1e12 / peak_tf, "reps": reps,
           "what": f"the whole AF (2N-1 = {2 * N - 1} delays x {M} Doppler bins) of {Bb} codes, Ahat written "
                   "as fp32 [B][2N-1][M]; output larger than L2"}
    del out
    torch.cuda.empty_cache()
    return res


def fp64_errors(g, x, out8, grad, dev):
    """Errors against the FP64 oracle, stated per configuration: the LFM
    chirp (N = 64, M = 128, all 127 delays, eps 1e-12) cell by cell, and on
    the benchmark batch the loss scalars of code 0 and 2048 sampled AF cells
    of codes 0 and 255 (the gradient of code 0 is added when the CPU baseline
    covers its whole AF)."""
    import numpy as np
    import torch

    import oracle
    from paper_2506_22935_gb300 import inputs
    res = {}
    phi = inputs.lfm_phases(64)
    w1 = g.Window.full(64, 128)
    A = g.af_forward(torch.from_numpy(phi).to(dev), 128, w1, 1e-12).cpu().numpy()[0]
    want = oracle.af_ahat(oracle.signal_from_phase(phi.astype(np.float64)), 128, *w1.as_tuple()[:4], 1e-12)
    res["lfm_N64_M128"] = {"ahat_max_abs": float(np.abs(A - want).max()),
                           "ahat_rms": float(np.sqrt(np.mean((A - want) ** 2))), "cells": int(A.size)}
    rng = np.random.default_rng(1)
    errs = []
    sub = [0, x.shape[0] - 1]
    Af = g.af_forward(x[sub], M, g.Window.full(N, M), EPS).cpu().numpy()
    for i, b in enumerate(sub):
        ks = rng.integers(-(N - 1), N, 1024)
        ms = rng.integers(-(M // 2), M // 2, 1024)
        s = oracle.signal_from_phase(x[b].double().cpu().numpy())
        want = oracle.af_cells(s, M, ks, ms, EPS)
        errs.append(np.abs(Af[i][ks + N - 1, ms + M // 2] - want))
    errs = np.concatenate(errs)
    o8 = out8[0].double().cpu().numpy()
    ref = oracle.loss(oracle.signal_from_phase(x[0].double().cpu().numpy()), M, oracle.full_window(N, M), 1.0, 1.0,
                      BETA, EPS)
    res["headline_B256_N1024_M2048"] = {
        "ahat_max_abs_sampled": float(errs.max()), "ahat_rms_sampled": float(np.sqrt(np.mean(errs ** 2))),
        "cells_sampled": int(errs.size),
        "loss_rel_wave0": {nm: float(abs(o8[i] - ref[i]) / abs(ref[i])) for i, nm in
                           ((0, "L"), (1, "PSL_soft"), (2, "ISL"), (3, "PSL_hard"))}}
    return res


def cufft_loss_grad(phi, N_len, M_len, box_m, beta, eps, chunk=64):
    """The comparison pipeline: the same loss and dL/dphi with every row DFT
    and its adjoint done by cuFFT (torch.fft) and the rest in eager torch ops.
    The gradient is written out with the split of the cell adjoint the
    kernels use -- w (1 + p) = w_b A' + [(w - w_b) A' + w (p - p0)], p =
    exp(beta (A2 - PSL)), p0 = exp(-beta PSL), A' = 1 + p0, w_b the weight of
    rows whose every bin carries the same weight -- because the row-uniform
    part contributes exactly nothing to dL/dphi; only the remainder goes
    through the inverse FFT (an FP32 chain rule through the whole cell
    adjoint loses the gradient to cancellation).
    phi [B, Nmax] fp32 (columns >= N_len[b] ignored), N_len [B] int64 tensor,
    one M for all.  Rows k >= 0 only, weight 2 for k > 0 (the mirror rows),
    Omega = every cell minus {k = 0, |m| <= box_m} (box_m an int or a [B]
    tensor).  Returns (L [B], dL/dphi)."""
    import torch
    F = torch.nn.functional
    dev = phi.device
    Bn, Nmax = phi.shape
    k = torch.arange(Nmax, device=dev)
    n = torch.arange(M_len, device=dev)
    mb = torch.minimum(n, M_len - n)
    box = torch.as_tensor(box_m, device=dev).expand(Bn)
    # q[k, p + k] for p < Nmax: row k shifted left by k
    shift = (torch.arange(Nmax, device=dev)[None, :] + k[:, None]).clamp(max=M_len - 1)
    losses, grads = [], []
    for c0 in range(0, Bn, chunk):
        p = phi[c0:c0 + chunk]
        C = p.shape[0]
        nl = N_len[c0:c0 + chunk]
        live = (k[None, :] < nl[:, None])
        s = torch.polar(live.float(), p)
        s_pad = F.pad(s, (0, M_len - Nmax))
        # row k of the lagged signal s[n - k] as a window of s with Nmax - 1
        # leading zeros (window Nmax - 1 - k), rows put back in k order
        s_ext = F.pad(s_pad, (Nmax - 1, 0))
        lag = s_ext.unfold(-1, M_len, 1).flip(1)
        R = s_pad[:, None, :] * torch.conj(lag)
        X = torch.fft.fft(R, dim=-1)
        E2 = ((s.real ** 2 + s.imag ** 2).sum(dim=1) ** 2)[:, None, None]
        A2 = (X.real ** 2 + X.imag ** 2 + eps) / E2
        w = torch.where(k[None, :, None] == 0, 1.0, 2.0) * (k[None, :, None] < nl[:, None, None])
        w = w * ~((k[None, :, None] == 0) & (mb[None, None, :] <= box[c0:c0 + C, None, None]))
        isl = (w * A2).sum(dim=(1, 2))
        psl = torch.logsumexp(beta * A2 + torch.log(w), dim=(1, 2)) / beta
        losses.append(psl + isl)
        p0 = torch.exp(-beta * psl)[:, None, None]
        wb = torch.where(k[None, :, None] == 0, torch.zeros_like(w), w)  # rows k >= 1 are uniform
        c = (w - wb) * (1.0 + p0) + w * p0 * torch.expm1(beta * A2)
        GR = torch.fft.ifft(c * X / E2, dim=-1) * M_len   # the adjoint DFT of each row
        q = (GR * torch.conj(R)).imag                    # Im(G_R conj(R))
        del R, X, GR
        t2 = torch.gather(q, 2, shift[None].expand(C, -1, -1)).sum(dim=1)
        grads.append(2.0 * (q.sum(dim=1)[:, :Nmax] - t2) * live)
        del q
    return torch.cat(losses), torch.cat(grads)


def time_cufft(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, out


def _timed_events(fn, steps, warmup, stream, flush=None):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps


def run_optim(args):
    """Masked-ISL phase optimisation: 64 random codes, N = 4096, M = 8192,
    window |k| <= 512, |m| <= 256 minus the origin, ISL loss, 500 Adam steps
    (lr 1e-2) captured in one CUDA graph and replayed."""
    import numpy as np
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs
    from paper_2506_22935_gb300.optim import Adam, PhaseOptimizer

    g.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    B3, N3, M3, K3, W3, STEPS = 64, 4096, 8192, 512, 256, 500
    phi0 = torch.from_numpy(inputs.random_phases(2506229350 + 3, B3, N3)).to(dev)
    phi = phi0.clone()
    opt = PhaseOptimizer(phi, M3, g.Window.masked(K3, W3), g.Loss(0.0, 1.0, BETA, EPS), Adam(lr=1e-2),
                         history_len=STEPS)
    opt.capture(STEPS)
    runs = max(1, args.optim_runs)

    def graph_run():
        opt.reset(phi0)
        opt.run(STEPS, graph=True)

    with ClockSampler(torch.device('cuda', 0)) as clk:
        ms_graph = _timed_events(graph_run, runs, 1, stream)
    hist = opt.history.cpu().numpy()
    ms_eager = _timed_events(lambda: (opt.reset(phi0), opt.run(STEPS, graph=False)), 1, 1, stream)
    rows = 2 * K3 + 1
    alg_step = B3 * 2 * rows * 5.0 * M3 * math.log2(M3)
    exe_step = B3 * 2 * (K3 + 1) * 5.0 * M3 * math.log2(M3)   # both transforms of the rows k >= 0
    peak, peak_src = _fp32_peak(dev)
    achieved = alg_step * STEPS / (ms_graph / 1e3) / 1e12
    cpu, errors = None, None
    if not args.no_cpu_baseline:
        import oracle
        s = oracle.signal_from_phase(phi0[0].cpu().numpy().astype(np.float64))
        win = (-K3, K3, -W3, W3, 0, 0)
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        _, gp_ref, o8_ref = oracle.grad(s, M3, win, 0.0, 1.0, BETA, EPS, nthreads=cores)
        dt = time.perf_counter() - t0
        o8_0, g_0 = g.af_loss_backward(phi0[:1], M3, g.Window.masked(K3, W3), g.Loss(0.0, 1.0, BETA, EPS))
        torch.cuda.synchronize()
        g_0 = g_0[0].double().cpu().numpy()
        errors = {"code0_step0_grad_rel_l2": float(np.linalg.norm(g_0 - gp_ref) / np.linalg.norm(gp_ref)),
                  "code0_step0_isl_rel": float(abs(float(o8_0[0, 2]) - o8_ref[2]) / o8_ref[2])}
        cpu = {"value": dt * B3 * STEPS * 1e3, "unit": "ms per run (extrapolated)", "cores": cores,
               "kind": "oracle", "sample": f"one FP64 loss + gradient of 1 of {B3} codes ({dt:.1f} s), "
                                           f"x {B3} codes x {STEPS} steps, Adam update not counted"}
    line = {"metric": "masked-ISL Adam run, 500 steps in one CUDA graph", "value": ms_graph,
            "unit": "ms per run", "higher_is_better": False, "n_gpus": 1, "steps": runs, "warmup": 1,
            "ms_per_step": ms_graph / STEPS, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B3} random codes, N={N3}, M={M3}, |k|<={K3}, |m|<={W3} minus origin, "
                                   f"ISL, Adam lr 1e-2, {STEPS} steps", "seed": 2506229350 + 3,
                       "l2": "working set (phases, moments, gradient partials) stays resident across steps"},
            "eager_ms_per_run": ms_eager,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "algorithmic_flop_per_step": alg_step, "executed_flop_per_step": exe_step,
                         "executed_frac": achieved * exe_step / alg_step / peak,
                         "peak_source": peak_src},
            "isl_median_start": float(np.median(hist[0])), "isl_median_end": float(np.median(hist[-1])),
            "cpu_baseline": cpu, "errors_vs_fp64": errors, "gpu_launches": 5 * STEPS * runs,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_ragged(args):
    """1000 codes of uneven length N_i log-uniform on [128, 8192], M_i = the
    next power of two >= 2 N_i, PSL(beta = 50) + ISL over every delay and
    Doppler bin minus the zero-delay mainlobe, fused loss + gradient."""
    import numpy as np
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs

    g.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    t_start = time.perf_counter()
    say = lambda what: print(f"[ragged {time.perf_counter() - t_start:7.1f} s] {what}", file=sys.stderr, flush=True)
    seed = 2506229350 + 4
    Ns = inputs.uneven_lengths(seed, 1000).astype(np.int64)
    Ms = np.array([1 << int(math.ceil(math.log2(2 * n))) for n in Ns], dtype=np.int64)
    phi_h = inputs.random_phases(seed + 1, 1, int(Ns.sum()))[0]
    x = torch.from_numpy(phi_h).to(dev)
    cells = float(((2 * Ns - 1) * Ms).sum())
    alg = float((2 * (2 * Ns - 1) * 5.0 * Ms * np.log2(Ms)).sum())
    exe = float((2 * Ns * 5.0 * Ms * np.log2(Ms)).sum())   # both transforms of the rows k >= 0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    loss = g.Loss(1.0, 1.0, BETA, EPS)
    plan = g.BatchPlan(Ns.astype(np.int32), losses=[loss], device=dev)
    out8 = torch.empty((1000, 8), dtype=torch.float32, device=dev)
    grad = torch.empty_like(x)
    steps = max(3, min(args.steps, 50))

    def plan_step():
        plan.loss_backward(x, out8=out8, grad=grad)

    say("plan created")
    ms_default = _timed_events(plan_step, steps, 3, stream, flush)
    say(f"untuned plan {ms_default:.2f} ms/step")
    cache = os.path.join(tempfile.gettempdir(), "graf_autotune_ragged.txt")
    plan.autotune(x, cache_path=cache)
    with ClockSampler(torch.device('cuda', 0)) as clk:
        ms_tuned = _timed_events(plan_step, steps, 3, stream, flush)
    info = plan.info()
    torch.cuda.synchronize()
    say(f"tuned plan {ms_tuned:.2f} ms/step")
    ref8, refg = out8.clone(), grad.clone()

    # per-M buckets, each padded to its longest code: one graf_af_loss_backward per bucket
    offs = np.concatenate([[0], np.cumsum(Ns)])
    buckets = []
    for Mb in sorted(set(Ms.tolist())):
        ids = np.nonzero(Ms == Mb)[0]
        nmax = int(Ns[ids].max())
        xs = np.zeros((len(ids), nmax), dtype=np.complex64)
        for j, b in enumerate(ids):
            xs[j, :Ns[b]] = np.exp(1j * phi_h[offs[b]:offs[b + 1]].astype(np.float64))
        xd = torch.from_numpy(xs.view(np.float32).reshape(len(ids), 2 * nmax)).to(dev)
        w = g.Window.full(nmax, Mb)
        nb = g.graf_af_backward_workspace_bytes(len(ids), nmax, Mb, w.c())
        buckets.append((Mb, ids, nmax, xd, w, torch.empty(nb, dtype=torch.uint8, device=dev),
                        torch.empty((len(ids), 8), dtype=torch.float32, device=dev),
                        torch.empty((len(ids), 2 * nmax), dtype=torch.float32, device=dev)))

    def padded_step():
        for Mb, ids, nmax, xd, w, ws, o8, gs in buckets:
            st = g.graf_af_loss_backward(xd.data_ptr(), g.GRAF_IN_COMPLEX, len(ids), nmax, Mb, w.c(), loss.c(),
                                         o8.data_ptr(), None, gs.data_ptr(), None, ws.data_ptr(), ws.numel(),
                                         stream.cuda_stream)
            assert st == 0, g.graf_status_string(st)

    say("padded buckets set up")
    ms_padded = _timed_events(padded_step, steps, 3, stream, flush)
    say(f"padded launches {ms_padded:.2f} ms/step")
    del buckets
    torch.cuda.empty_cache()

    cmp = None
    if not args.no_cufft:
        parts = []
        sample = np.arange(0, 1000, args.cufft_stride)
        for Mb in sorted(set(Ms[sample].tolist())):
            ids = sample[Ms[sample] == Mb]
            nmax = int(Ns[ids].max())
            ph = np.zeros((len(ids), nmax), dtype=np.float32)
            for j, b in enumerate(ids):
                ph[j, :Ns[b]] = phi_h[offs[b]:offs[b + 1]]
            chunk = max(1, (1 << 30) // (nmax * Mb * 8))
            parts.append((torch.from_numpy(ph).to(dev), torch.from_numpy(Ns[ids]).to(dev), Mb,
                          torch.from_numpy(np.maximum(Mb // Ns[ids] - 1, 0)).to(dev), chunk, ids))

        def cufft_step():
            return [cufft_loss_grad(ph, nl, Mb, box, BETA, EPS, chunk=ch) for ph, nl, Mb, box, ch, _ in parts]

        ms_c, res = time_cufft(cufft_step, 1, 0, stream)
        say(f"cuFFT pipeline {ms_c:.1f} ms/step")
        lc_ = torch.empty(1000, device=dev)
        for (ph, nl, Mb, box, ch, ids), (l_, _) in zip(parts, res):
            lc_[torch.from_numpy(ids).to(dev)] = l_
        s_cells = float(((2 * Ns[sample] - 1) * Ms[sample]).sum())
        sl = torch.from_numpy(sample).to(dev)
        cmp = {"value": s_cells / (ms_c / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms_c,
               "sample": f"every {args.cufft_stride}th code ({len(sample)} codes, {s_cells:.3g} cells), one pass",
               "loss_max_rel_diff": float(((lc_[sl] - ref8[sl, 0]).abs() / ref8[sl, 0].abs()).max()),
               "what": "per-M buckets padded to the longest code, torch.fft (cuFFT) + eager torch ops + autograd"}
        del res, parts
        torch.cuda.empty_cache()
    errors = None
    if not args.no_cpu_baseline:
        import oracle
        o8h, gh = ref8.cpu().numpy(), refg.cpu().numpy()
        errors = {}
        for Mb in sorted(set(Ms.tolist())):
            if Mb > 8192:  # the M = 16384 bucket's shortest code costs ~3 min of oracle time: in the slow test
                continue
            ids = np.nonzero(Ms == Mb)[0]
            b = int(ids[np.argmin(Ns[ids])])
            n = int(Ns[b])
            sb = oracle.signal_from_phase(phi_h[offs[b]:offs[b + 1]].astype(np.float64))
            _, gp, o8r = oracle.grad(sb, Mb, oracle.full_window(n, Mb), 1.0, 1.0, BETA, EPS)
            gb = gh[offs[b]:offs[b + 1]].astype(np.float64)
            errors[f"M{Mb}_N{n}"] = {"grad_rel_l2": float(np.linalg.norm(gb - gp) / np.linalg.norm(gp)),
                                     "loss_rel": float(abs(o8h[b, 0] - o8r[0]) / abs(o8r[0]))}
        say("oracle checks done")
    plan.close()
    peak, peak_src = _fp32_peak(dev)
    achieved = alg / (ms_tuned / 1e3) / 1e12
    line = {"metric": "ragged-batch AF fwd+bwd Gcells/s", "value": cells / (ms_tuned / 1e3) / 1e9,
            "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "steps": steps, "warmup": 3,
            "ms_per_step": ms_tuned, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "1000 random codes, N_i log-uniform on [128, 8192], M_i = nextpow2(2 N_i), "
                                   "all delays and Doppler bins minus the zero-delay mainlobe, PSL(beta=50)+ISL, "
                                   "loss + gradient w.r.t. phases", "seed": seed, "cells_per_step": cells,
                       "l2": "flushed between steps (256 MB write, outside the timed events)"},
            "untuned_plan_ms": ms_default, "padded_per_M_launches_ms": ms_padded,
            "plan": info,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "algorithmic_flop_per_step": alg,
                         "executed_flop_per_step": exe, "executed_frac": achieved * exe / alg / peak,
                         "peak_source": peak_src},
            "cufft_pipeline": cmp, "clocks": clk.summary(),
            "errors_vs_fp64": errors, "errors_note": "the shortest code of each M bucket up to 8192 against the "
                                                     "FP64 oracle (every bucket up to 16384 in the slow GPU test)"}
    print(json.dumps(line), flush=True)


def run_periodic(args):
    """The paper's own periodic AF (Eq. 7, +j exponent) at its experiments'
    length N = 256 (Sec. 7.1.2): 4096 random polyphase codes, all N delays x N
    Doppler bins minus the origin, PSL(beta = 50) + ISL, loss + gradient
    w.r.t. the phases."""
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs

    g.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Bp, Np = args.pbatch, 256
    seed = 2506229350 + 6
    x = torch.from_numpy(inputs.random_phases(seed, Bp, Np)).to(dev)
    w, loss = g.Window.periodic(Np), g.Loss(1.0, 1.0, BETA, EPS)
    nb = g.graf_paf_workspace_bytes(Bp, Np, w.c())
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out8 = torch.empty((Bp, 8), dtype=torch.float32, device=dev)
    grad = torch.empty((Bp, Np), dtype=torch.float32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        st = g.graf_paf_loss_backward(x.data_ptr(), g.GRAF_IN_PHASE, Bp, Np, 1, w.c(), loss.c(), out8.data_ptr(),
                                      None, None, grad.data_ptr(), ws.data_ptr(), nb, stream.cuda_stream)
        assert st == 0, g.graf_status_string(st)

    steps = max(3, min(args.steps, 100))
    with ClockSampler(torch.device('cuda', 0)) as clk:
        ms = _timed_events(step, steps, 5, stream, flush)
    cells = Bp * Np * Np
    alg = Bp * 2 * Np * 5.0 * Np * math.log2(Np)   # forward + adjoint DFT of every delay row
    exe = Bp * 2 * (Np // 2 + 1) * 5.0 * Np * math.log2(Np)   # rows 0..N/2 (row N - k mirrors row k)
    peak, peak_src = _fp32_peak(dev)
    achieved = alg / (ms / 1e3) / 1e12
    chi = g.paf_forward(x[:64], 1, normalise=True)
    torch.cuda.synchronize()
    import numpy as np

    import oracle
    s0 = oracle.signal_from_phase(x[0].double().cpu().numpy())
    _, gp, o8r = oracle.pgrad(s0, w.as_tuple(), 1.0, 1.0, BETA, EPS, sign=1)
    chi_ref = oracle.paf_chi(s0, 1, normalise=True)
    g0 = grad[0].double().cpu().numpy()
    errors = {"code0_grad_rel_l2": float(np.linalg.norm(g0 - gp) / np.linalg.norm(gp)),
              "code0_loss_rel": float(abs(float(out8[0, 0]) - o8r[0]) / abs(o8r[0])),
              "code0_chi_max_abs": float(np.abs(chi[0].double().cpu().numpy() - chi_ref).max())}
    line = {"metric": "periodic AF fwd+bwd Gcells/s at N=256", "value": cells / (ms / 1e3) / 1e9,
            "unit": UNIT, "higher_is_better": True, "n_gpus": 1, "steps": steps, "warmup": 5,
            "ms_per_step": ms, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{Bp} random polyphase codes, periodic AF (Eq. 7, +j), N={Np}, "
                                   "all delays and Doppler bins minus the origin, PSL(beta=50)+ISL, "
                                   "loss + gradient w.r.t. phases", "seed": seed,
                       "l2": "flushed between steps (256 MB write, outside the timed events)"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "algorithmic_flop_per_step": alg,
                         "executed_flop_per_step": exe, "executed_frac": achieved * exe / alg / peak,
                         "peak_source": peak_src},
            "mean_psl_hard": float(out8[:, 3].mean()), "mean_chi_max": float(chi.amax(dim=(1, 2)).mean()),
            "errors_vs_fp64": errors, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_lpi(args):
    """The paper's experiment (Sec. 7.1): L = PSL + lambda alpha SV (Eq. 25),
    alpha = 2000, periodic AF of Eq. 7, N = 256 phase codes, Adam lr 0.01,
    2000 iterations; PSL the hard maximum of Ahat^2 over every cell but the
    origin (Eq. 18, differentiated through its arg-max cell).  64 random codes
    per lambda, each lambda's 2000 steps captured in one CUDA graph."""
    import numpy as np
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs
    from paper_2506_22935_gb300.optim import Adam, PhaseOptimizer

    g.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Bl, Nl, STEPS, ALPHA, BETA_L = 64, 256, 2000, 2000.0, math.inf
    seed = 2506229350 + 7
    phi0 = torch.from_numpy(inputs.random_phases(seed, Bl, Nl)).to(dev)
    win = g.Window.periodic(Nl)
    res = {}
    with ClockSampler(torch.device('cuda', 0)) as clk:
        for lam in (0.0, 0.5, 1.0, 2.0):
            phi = phi0.clone()
            opt = PhaseOptimizer(phi, window=win, loss=g.Loss(1.0, 0.0, BETA_L, EPS), adam=Adam(lr=1e-2),
                                 history_len=STEPS, periodic_sign=1, spectral_weight=lam * ALPHA)
            opt.capture(STEPS)
            opt.reset(phi0)
            opt.run(STEPS)                        # warm-up run
            opt.reset(phi0)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            opt.run(STEPS)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            out8 = torch.empty((Bl, 8), device=dev)
            o8, _ = g.paf_loss_backward(phi, win, g.Loss(1.0, 0.0, BETA_L, EPS), 1)
            sv, _ = g.spectral_variance(phi, 1.0)
            sv0, _ = g.spectral_variance(phi0, 1.0)
            hist = opt.history.cpu().numpy()
            conv = int(np.median(np.argmax(hist <= hist[-1][None, :] * 1.01 + 1e-12, axis=0)))
            psl = o8[:, 3].cpu().numpy()
            res[str(lam)] = {"ms_per_run": ms, "ms_per_step": ms / STEPS,
                             "median_psl_hard": float(np.median(psl)),
                             "median_psl_db": float(np.median(10 * np.log10(psl))),
                             "median_spectral_variance": float(sv.median()),
                             "median_spectral_variance_start": float(sv0.median()),
                             "median_final_loss": float(np.median(hist[-1])),
                             "median_step_within_1pct_of_final": conv}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        oracle.optimize_experiment(phi0[0].cpu().numpy().astype(np.float64), win.as_tuple(), 1.0, 0.0, BETA_L,
                                   EPS, 0.5 * ALPHA, 3)
        dt = (time.perf_counter() - t0) / 3
        cpu = {"value": dt * STEPS * 1e3, "unit": "ms per code-run (extrapolated)", "cores": 1, "kind": "oracle",
               "sample": f"3 FP64 steps of one code ({dt * 1e3:.0f} ms each) x {STEPS} steps"}
    v = res["0.5"]["ms_per_run"] / Bl
    line = {"metric": "experiment run (Sec. 7.1): 2000 Adam steps of PSL + lambda alpha SV, N = 256",
            "value": v, "unit": "GPU ms per code-run at lambda = 0.5 (64 codes per graph)",
            "higher_is_better": False, "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{Bl} random codes per lambda, periodic AF (Eq. 7, +j), N={Nl}, "
                                   f"alpha={ALPHA:.0f}, hard PSL (Eq. 18), Adam lr 1e-2, {STEPS} steps",
                       "seed": seed},
            "vs_paper": {"paper_seconds_per_run_lambda_0.5_cpu": 67.0,
                         "paper_spectral_variance": {"0": 2.02e-5, "0.5": 3.03e-6, "2": 8.02e-7}},
            "lambda": res, "cpu_baseline": cpu, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_terms(args):
    """The composite and multi-scenario terms at the benchmark size (256 codes,
    N = 1024, M = 2048): mainlobe width + modulus variance (Sec. 5.1, Eq. 22),
    the target match over the whole AF (Eq. 22), and a three-scenario plan
    (Eq. 24: the whole AF with PSL + ISL, a range-Doppler box with ISL, a
    velocity band with PSL + ISL) with loss and summed gradient."""
    import numpy as np
    import torch

    from paper_2506_22935_gb300 import graf as g
    from paper_2506_22935_gb300 import inputs

    g.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    x = torch.from_numpy(inputs.random_phases(SEED + 20, B, N)).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    grad = torch.empty((B, N), device=dev)
    out8 = torch.zeros((B, 8), device=dev)
    terms = torch.empty((B, 2), device=dev)
    steps = max(3, min(args.steps, 50))
    res = {}

    def comp():
        st = g.graf_composite_terms(x.data_ptr(), g.GRAF_IN_PHASE, B, N, 50.0, EPS, 1.0, 1.0, out8.data_ptr(),
                                    terms.data_ptr(), None, grad.data_ptr(), 1, sp)
        assert st == 0, g.graf_status_string(st)

    ms = _timed_events(comp, steps, 3, stream, flush)
    res["composite_width_modvar"] = {"ms": ms, "codes_per_s": B / (ms / 1e3)}
    w = g.Window.full(N, M, k_ml=-1, m_ml=-1)
    target = torch.zeros((B, 2 * N - 1, M), device=dev)  # 4.3 GB: a sidelobe-free ideal
    nb = g.graf_af_match_workspace_bytes(B, N, M, w.c())
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    loss = torch.empty(B, device=dev)

    def match():
        st = g.graf_af_match(x.data_ptr(), g.GRAF_IN_PHASE, B, N, M, w.c(), target.data_ptr(), 1.0, EPS,
                             loss.data_ptr(), None, None, grad.data_ptr(), 0, ws.data_ptr(), nb, sp)
        assert st == 0, g.graf_status_string(st)

    ms = _timed_events(match, steps, 3, stream, flush)
    cells = B * (2 * N - 1) * M
    res["match_full_af"] = {"ms": ms, "Gcells_per_s": cells / (ms / 1e3) / 1e9,
                            "target_GB_per_s": target.numel() * 4 / (ms / 1e3) / 1e9}
    del target, ws
    torch.cuda.empty_cache()
    src = np.repeat(np.arange(B), 3)
    windows, losses = [], []
    for i in range(3 * B):
        if i % 3 == 0:
            windows.append(g.Window.full(N, M))
            losses.append(g.Loss(1.0, 1.0, BETA, EPS))
        elif i % 3 == 1:
            windows.append(g.Window(-256, 256, -128, 128, 0, 0))
            losses.append(g.Loss(0.0, 1.0, BETA, EPS))
        else:
            windows.append(g.Window(-(N - 1), N - 1, 64, 512, -1, -1))
            losses.append(g.Loss(0.5, 1.0, BETA, EPS))
    plan = g.BatchPlan.scenarios([N] * B, src, windows, losses, M=[M] * (3 * B))
    lam = torch.tensor([1.0, 0.5, 0.25] * B, device=dev)
    o8 = torch.empty((3 * B, 8), device=dev)
    gsum = torch.empty(B * N, device=dev)
    xs = x.reshape(-1)

    def scen():
        plan.loss_backward(xs, dL=lam, out8=o8, grad=gsum)

    ms = _timed_events(scen, steps, 3, stream, flush)
    res["scenarios_3_per_code"] = {"ms": ms, "codes_per_s": B / (ms / 1e3),
                                   "plan": plan.info()}
    plan.close()
    line = {"metric": "composite and multi-scenario terms at N=1024 M=2048", "value": res["match_full_af"]["Gcells_per_s"],
            "unit": "Gcells/s (target match over the whole AF, fwd+bwd)", "higher_is_better": True, "n_gpus": 1,
            "steps": steps, "warmup": 3, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{B} random codes, N={N}, M={M}", "l2": "flushed between steps"},
            "terms": res}
    print(json.dumps(line), flush=True)


def learned_eval(args, dev):
    """The learned half of the metric (the NN -> waveform -> GRAF -> loss
    pipeline of Sec. 6.1): labels = each training spec's own loss optimised on
    the GPU from one common seeded code; the MLP trained on (spec, label)
    pairs with the phase label loss; then, as a second arm, fine-tuned end to
    end through the GRAF layer on the masked ISL.  Each arm: the median over
    held-out specs of the GPU time to the spec's masked-ISL target from the
    proposal over that from a random initialisation (learned.time_to_target,
    CUDA events per step)."""
    import numpy as np
    import torch

    from paper_2506_22935_gb300 import inputs, learned
    t_all = time.perf_counter()
    train = inputs.design_specs(SEED + 10, args.train_specs)
    test = inputs.design_specs(SEED + 11, args.test_specs)
    net = learned.ProposalMLP(seed=SEED, lr=args.mlp_lr, device=dev)
    secs, label_curve, graf_curve = {}, [], []
    t0 = time.perf_counter()
    init = (learned.lfm_init(args.train_specs) if args.label_init == "lfm"
            else learned.common_init(args.train_specs, SEED + 12))
    codes, lh = learned.optimise_codes(train, init, args.label_steps, isl_only=bool(args.label_isl_only),
                                       device=dev)
    secs["labels"] = time.perf_counter() - t0
    feats = torch.from_numpy(inputs.spec_features(train)).to(dev)
    tgt = torch.from_numpy(codes).to(dev)
    loss = torch.empty(args.batch_mlp, device=dev)
    rng = np.random.default_rng(0)
    t1 = time.perf_counter()
    for _ in range(args.label_epochs):
        order = torch.from_numpy(rng.permutation(args.train_specs)).to(dev)
        for i in range(0, args.train_specs - args.batch_mlp + 1, args.batch_mlp):
            net.train_step(feats[order[i:i + args.batch_mlp]], tgt[order[i:i + args.batch_mlp]], loss_out=loss)
        label_curve.append(float(loss.mean()))
    torch.cuda.synchronize(dev)
    secs["label_train"] = time.perf_counter() - t1
    t2 = time.perf_counter()
    target = learned.masked_isl_targets(test, args.eval_steps, device=dev)
    rand = learned.random_run(test, args.eval_steps, device=dev)
    secs["targets_and_random_run"] = time.perf_counter() - t2

    def arm(r):
        sl, sr = r["steps_learned"], r["steps_random"]
        ratio = r["time_learned_ms"] / r["time_random_ms"]
        return {"value": float(np.median(ratio)),
                "learned_wins_fraction": float(np.mean(ratio < 1.0)),
                "learned_reached_fraction": float(np.mean(sl <= args.eval_steps)),
                "random_reached_fraction": float(np.mean(sr <= args.eval_steps)),
                "median_steps_learned": float(np.median(sl)), "median_steps_random": float(np.median(sr)),
                "median_ms_learned": float(np.median(r["time_learned_ms"])),
                "median_ms_random": float(np.median(r["time_random_ms"])),
                "median_isl0_learned": float(np.median(r["isl0_learned"])),
                "median_isl0_random": float(np.median(r["isl0_random"])),
                "mlp_inference_ms": r["mlp_ms"], "run_ms_learned": r["run_ms_learned"],
                "run_ms_random": r["run_ms_random"]}

    labels_arm = arm(learned.time_to_target(net, test, target, rand, args.eval_steps, device=dev))
    tuned = None
    if args.graf_epochs > 0:
        t3 = time.perf_counter()
        trainer = learned.GrafTrainer(net, train, group=args.batch_mlp, isl_only=args.train_isl_only)
        for _ in range(args.graf_epochs):
            graf_curve.append(trainer.epoch())
        torch.cuda.synchronize(dev)
        trainer.close()
        secs["graf_train"] = time.perf_counter() - t3
        tuned = arm(learned.time_to_target(net, test, target, rand, args.eval_steps, device=dev))
    secs["total"] = time.perf_counter() - t_all
    errors = None
    if not args.no_cpu_baseline:
        # the trained network's outputs and one held-out spec's masked-ISL loss
        # and gradient at its proposal, against the FP64 references
        import oracle
        from oracle import mlp as omlp

        from paper_2506_22935_gb300 import graf as g
        nchk = min(16, args.test_specs)
        sub = {k: v[:nchk] for k, v in test.items()}
        fsub = inputs.spec_features(sub)
        out = net.forward(torch.from_numpy(fsub).to(dev)).cpu().numpy().astype(np.float64)
        ref, _ = omlp.forward(fsub.astype(np.float64), net.master.cpu().numpy().astype(np.float64))
        i = int(np.argmin(sub["K"]))  # the narrowest delay mask: the cheapest FP64 check
        phi_i = np.mod(out[i], 2 * np.pi).astype(np.float32)
        win = g.Window.masked(int(sub["K"][i]), int(sub["Mw"][i]))
        plan = g.BatchPlan([1024], M=[2048], windows=[win], losses=[g.Loss(0.0, 1.0, 50.0, EPS)], device=dev)
        o8, gr = plan.loss_backward(torch.from_numpy(phi_i).to(dev))
        torch.cuda.synchronize(dev)
        plan.close()
        _, gp_ref, o8_ref = oracle.grad(oracle.signal_from_phase(phi_i.astype(np.float64)), 2048, win.as_tuple(),
                                        0.0, 1.0, 50.0, EPS, nthreads=os.cpu_count() or 1)
        gr = gr.double().cpu().numpy()
        errors = {"mlp_output_rel_l2_vs_bf16_reference": float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
                  "mlp_specs_checked": nchk,
                  "masked_isl_rel": float(abs(float(o8[0, 2]) - o8_ref[2]) / o8_ref[2]),
                  "masked_isl_grad_rel_l2": float(np.linalg.norm(gr - gp_ref) / np.linalg.norm(gp_ref)),
                  "graf_check": f"held-out spec {i} (K={int(sub['K'][i])}, Mw={int(sub['Mw'][i])}) at its proposal"}
    every = lambda c: [round(x, 4) for x in c[:: max(1, len(c) // 10)]]
    return {"metric": "time to masked-ISL target, learned vs plain", "value": labels_arm["value"],
            "unit": "median over held-out specs of GPU time to target, learned proposal / random init",
            "higher_is_better": False,
            "config": {"train_specs": args.train_specs, "test_specs": args.test_specs, "N": 1024, "M": 2048,
                       "labels": f"each training spec's own loss (w_psl PSL(beta=50) + w_isl ISL over its mask), "
                                 f"Adam lr 1e-2, {args.label_steps} steps from "
                                 + ("one common seeded random code" if args.label_init == "common"
                                    else "the discrete chirp"),
                       "label_epochs": args.label_epochs, "graf_finetune_epochs": args.graf_epochs,
                       "eval_steps": args.eval_steps,
                       "target": f"per held-out spec, the median masked ISL of 4 random initialisations after "
                                 f"{args.eval_steps} Adam steps",
                       "timing": "CUDA events after every optimiser step of the batched run; MLP inference timed"},
            "median_target_isl": float(np.median(target)),
            "label_isl_median_start_end": [float(np.median(lh[0])), float(np.median(lh[-1]))],
            "labels_only": labels_arm, "labels_then_graf_finetune": tuned,
            "label_loss_curve": every(label_curve), "graf_loss_curve": every(graf_curve), "seconds": secs,
            "errors_vs_fp64": errors}


def run_learned(args):
    """The learned half of the metric as a line of its own (see learned_eval)."""
    import torch

    from paper_2506_22935_gb300 import graf as g
    g.load()
    res = learned_eval(args, torch.device("cuda", 0))
    line = {"metric": res.pop("metric"), "value": res.pop("value"), "unit": res.pop("unit"),
            "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "bf16 mlp, f32 af", **res}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="graf", choices=["graf", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison pipeline")
    ap.add_argument("--no-forward-store", action="store_true", help="skip the full-AF forward store timing")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain time to target")
    ap.add_argument("--batch", type=int, default=B,
                    help="waveforms per GPU (default 256, the benchmark workload; smaller only for profiling)")
    ap.add_argument("--workload", default="af", choices=["af", "learned", "optim", "ragged", "periodic", "lpi",
                                                                 "terms"])
    ap.add_argument("--optim-runs", type=int, default=3)
    ap.add_argument("--pbatch", type=int, default=4096,
                    help="periodic workload: codes per step (default 4096; smaller only for profiling)")
    ap.add_argument("--cufft-stride", type=int, default=50,
                    help="ragged workload: the cuFFT comparison runs on every n-th code")
    ap.add_argument("--train-specs", type=int, default=20000)
    ap.add_argument("--test-specs", type=int, default=512)
    ap.add_argument("--label-steps", type=int, default=500)
    ap.add_argument("--label-epochs", type=int, default=60)
    ap.add_argument("--label-init", default="common", choices=["common", "lfm"])
    ap.add_argument("--label-isl-only", type=int, default=0)
    ap.add_argument("--graf-epochs", type=int, default=100)
    ap.add_argument("--train-isl-only", type=int, default=1)
    ap.add_argument("--batch-mlp", type=int, default=256)
    ap.add_argument("--mlp-lr", type=float, default=1e-3)
    ap.add_argument("--eval-steps", type=int, default=500)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "optim":
        run_optim(args)
    elif args.workload == "ragged":
        run_ragged(args)
    elif args.workload == "periodic":
        run_periodic(args)
    elif args.workload == "lpi":
        run_lpi(args)
    elif args.workload == "terms":
        run_terms(args)
    else:
        run_graf(args)


if __name__ == "__main__":
    main()
