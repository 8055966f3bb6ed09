"""Register budget of the one-wave image-strip kernels (CPU: nvcc only).

The 2048^2 image of 16 x 16 blocks runs as one wave of seven CTAs of 128
threads per SM, which leaves each thread at most 72 registers (65536 / 896,
rounded down to the allocation unit).  A change that pushes a direction of
the kernel past that, or makes it spill, costs the wave (a changed form of
the spectral direction once spilled 20 bytes a thread and ran at half speed;
no direction spills now), so the ptxas resource report of every direction is
checked here.
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_28519_gb300", "csrc")

# direction index of the template argument -> (max registers, max spill-load bytes)
LIMITS = {0: (72, 0), 1: (72, 0), 2: (72, 0), 3: (72, 0)}


def _ptxas_report(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
           "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-Xptxas", "-v", "-c", os.path.join(CSRC, "fp32_fused.cu"), "-o", str(tmp_path / "f.o")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def test_one_wave_strip_kernels_fit_seven_ctas_per_sm(tmp_path):
    report = _ptxas_report(tmp_path)
    found = {}
    # "Compiling entry function '<mangled k_strip16_waveILi<d>E...>'" followed by the
    # spill line and the "Used N registers" line of that function
    blocks = re.split(r"Compiling entry function '", report)
    for b in blocks[1:]:
        m = re.match(r"_ZN4bdct14k_strip16_waveILi(\d)EEEvNS_11FusedParamsE", b)
        if not m:
            continue
        d = int(m.group(1))
        regs = int(re.search(r"Used (\d+) registers", b).group(1))
        spill = re.search(r"(\d+) bytes spill loads", b)
        found[d] = (regs, int(spill.group(1)) if spill else 0)
    assert sorted(found) == [0, 1, 2, 3], found
    for d, (regs, spill) in found.items():
        max_regs, max_spill = LIMITS[d]
        assert regs <= max_regs, (d, regs)
        assert spill <= max_spill, (d, spill)
