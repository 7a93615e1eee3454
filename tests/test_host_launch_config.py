"""Host-side checks of the launch configuration the library derives, on the
CPU: the host mirrors of the row plan (threads per row, per CTA, row slots)
agree with the device-side RowPlan; the number of gradient accumulators per
CTA is a power of two no larger than the slot count, fits the opt-in shared
memory, and is the largest that its rule allows (two CTAs per SM where the
registers allow two and that costs at most two scatter turns, else the largest
that fits); row tiles are whole multiples of the slot count, cover the rows
exactly once, and are as large as possible while the grid still gives every SM
four CTAs.  The host program is compiled by nvcc as plain host code."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2506_22935_gb300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("launch_config")
    subprocess.check_call([sys.executable, os.path.join(CSRC, "gen_twiddles.py"), str(d / "twiddles.inc")])
    exe = d / "launch_config_host"
    src = os.path.join(ROOT, "tests", "host", "launch_config_host.cu")
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O2", "-I", CSRC, "-I",
                           os.path.join(ROOT, "include"), "-I", str(d), "-x", "cu", src, "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    rows = {}
    for line in out.splitlines():
        tag, *vals = line.split()
        rows.setdefault(tag, []).append([int(v) for v in vals])
    return rows


def test_host_mirrors_match_row_plan(dump):
    for M, tpr, threads, slots, min_blocks, h_tpr, h_threads, h_slots in dump["mirror"]:
        assert (h_tpr, h_threads, h_slots) == (tpr, threads, slots), M
        assert tpr * slots == threads and threads % 32 == 0 and threads <= 1024
        assert min_blocks in (1, 2)


def test_accumulator_copies_follow_their_rule(dump):
    (max_smem, smem_per_sm, _), = dump["const"]
    plan = {r[0]: r for r in dump["mirror"]}
    for M, N, real, per, copies, smem, smem2 in dump["acc"]:
        slots, min_blocks = plan[M][3], plan[M][4]
        case = (M, N, real, per)
        if copies == 0:  # unsupported: not even one accumulator fits
            assert smem > max_smem, case
            continue
        assert copies & (copies - 1) == 0 and copies <= slots, case
        assert smem <= max_smem, case
        if copies == slots:
            continue
        budget = smem_per_sm // min_blocks - 1024
        if min_blocks == 2 and 2 * copies >= slots and smem <= budget:
            assert smem2 > budget, case      # the largest within two CTAs per SM
        else:
            assert smem2 > max_smem, case    # the largest that fits at all


def test_row_tiles_cover_the_rows_and_fill_the_gpu(dump):
    (_, _, sms), = dump["const"]
    for B, M, lo, hi, slots, rpt, tiles in dump["tile"]:
        nrows, case = hi - lo + 1, (B, M, hi)
        rps_max = 16 if M >= 128 else 8
        assert rpt % slots == 0 and slots <= rpt <= rps_max * slots, case
        assert (tiles - 1) * rpt < nrows <= tiles * rpt, case
        # the most rows per slot that still gives every SM four CTAs
        if rpt > slots:
            assert B * tiles >= 4 * sms, case
        if rpt < rps_max * slots:
            assert B * -(-nrows // (2 * rpt)) < 4 * sms, case
