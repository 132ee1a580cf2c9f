"""The adjoint engine's schedule, checked on the host (no GPU): builds
tests/adjoint_schedule_check.cu with nvcc (lbm_adjoint.cu with its few
runtime calls replaced by stand-ins) and runs it over five tape structures in
FP32 and one in FP64 on periodic axes, and over walled axes (y; x and y) in
FP32 and FP64.  It checks slot bounds, storage of every plane read, the
staging of every operand and stencil tap in its phase, flushes, the walls'
ghost signs and bounce-back masks, and, when NVRTC is available, that the
generated level kernels (with the wall helpers) compile and that the
argument packs can be exchanged between reverse passes."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_adjoint_schedule_on_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "adjoint_schedule_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1812_02459_gb300", "csrc"),
                    os.path.join(HERE, "adjoint_schedule_check.cu"), "-o", exe, "-ldl"],
                   check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe, "1"], capture_output=True, text=True, timeout=600)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [l for l in r.stdout.splitlines() if "failures" in l]
    assert len(lines) == 9 and all(l.endswith("failures 0") for l in lines)
