"""Resources ptxas reports for the docking kernel's FP32 instantiations (nvcc cross-compiles for
sm_103a without a GPU, so this runs on the CPU).

They pin two properties the measured performance depends on:
  * the one-warp-per-item FP32 instantiations are the `dock_kernel_wide` entry point, at 96
    registers with nothing spilled (the fastest shape of the dominant FP32 bucket);
  * the 8-warps-per-item instantiations (the serving loop's shape for small batches) stay
    `dock_kernel` at 64 registers and use 2 named barriers.  Other ways of writing the two entry
    points compiled that kernel with all 16 barriers reserved, and small serving batches were 8%
    slower at the median although a lone ligand's launch did not change.
"""
import os
import re
import subprocess
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2209_05069_gb300 import build

ENTRY = re.compile(r"Compiling entry function '_ZN7dockgpu(\d+)(dock_kernel(?:_wide)?)ILi(\d+)ELi(\d+)ELi(\d+)ELi(\d+)E")
REGS = re.compile(r"Used (\d+) registers, used (\d+) barriers")
SPILL = re.compile(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads")


def _resources(gt, g, t):
    """{(entry, MAXN, GT, G, T): (registers, barriers, spill stores, spill loads)} of one unit."""
    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        cmd = [nvcc] + build.ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", build.INCLUDE, "-I", build.CSRC,
                                     f"-DDOCK_INST_GT={gt}", f"-DDOCK_INST_G={g}", f"-DDOCK_INST_T={t}", "-Xptxas", "-v",
                                     "-c", os.path.join(build.CSRC, "dock_kernels_inst.cu"), "-o", os.path.join(d, "k.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out, cur, spill = {}, None, None
    for line in r.stderr.splitlines():
        m = ENTRY.search(line)
        if m:
            cur, spill = (m.group(2),) + tuple(int(m.group(i)) for i in range(3, 7)), None
            continue
        m = SPILL.search(line)
        if m and cur:
            spill = (int(m.group(2)), int(m.group(3)))
        m = REGS.search(line)
        if m and cur:
            out[cur] = (int(m.group(1)), int(m.group(2))) + (spill or (0, 0))
            cur = None
    return out


@pytest.fixture(scope="module")
def fp32_units():
    with ThreadPoolExecutor(max_workers=2) as ex:
        wide, serve = ex.map(lambda a: _resources(*a), [(0, 1, 2), (0, 8, 1)])
    return wide, serve


def test_one_warp_per_item_fp32_is_the_wide_entry_point(fp32_units):
    wide, _ = fp32_units
    assert sorted(k[1] for k in wide) == [32, 64, 96, 128, 160]
    for (entry, maxn, gt, g, t), (regs, bars, st, ld) in wide.items():
        assert entry == "dock_kernel_wide", (maxn, gt, g, t)
        assert regs <= 96 and st == 0 and ld == 0, (maxn, regs, st, ld)


def test_serving_shape_keeps_the_launch_bound_and_two_barriers(fp32_units):
    _, serve = fp32_units
    assert sorted(k[1] for k in serve) == [32, 64, 96, 128, 160]
    for (entry, maxn, gt, g, t), (regs, bars, st, ld) in serve.items():
        assert entry == "dock_kernel", (maxn, gt, g, t)
        assert regs <= 64, (maxn, regs)
        assert bars == 2, (maxn, bars)
