"""Launch-plan invariants of the library, checked on the host (no GPU): the
plans of K1, K2, K2P and K3T and every configuration the autotuner may
install stay within the shared-memory and tensor-memory limits of one CTA,
keep every split-K range non-empty and every TMA inner extent 16-byte
aligned, and fit the scratch grom_create allocates (tests/plan_invariants.cpp,
linked against libgrom.so)."""
import os
import shutil
import subprocess

import pytest

import paper_2311_03694_gb300 as grom

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
    return inc if os.path.exists(os.path.join(inc, "cuda.h")) else None


def test_plan_invariants(tmp_path):
    lib = grom.build()
    inc = _cuda_include()
    if inc is None:
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path / "plan_invariants")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I" + inc, "-I" + os.path.join(ROOT, "paper_2311_03694_gb300", "csrc"),
                    os.path.join(HERE, "plan_invariants.cpp"), lib, "-Wl,-rpath," + os.path.dirname(lib), "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "0 failed" in r.stdout
