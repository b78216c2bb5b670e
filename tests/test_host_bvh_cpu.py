"""Host parts of the library on the CPU: tests/host/check_bvh.cpp against the
builder (every triangle in one leaf of the global BVH, closest hits equal to
brute force, grid cells reference every triangle that reaches into them,
packed vertices bit for bit), and tests/host/check_cache.cpp against the
subdomain-cache planner and the index relocation of a load (every traced cell
complete and alone in its part of the cache)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_06474_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_bvh_builder_against_brute_force(tmp_path):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers (vector types)")
    exe = tmp_path / "check_bvh"
    cmd = ["g++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", CUDA_INC,
           os.path.join(ROOT, "tests", "host", "check_bvh.cpp"), os.path.join(CSRC, "bvh_build.cpp"),
           "-o", str(exe), "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr


def test_cell_cache_planner_and_relocation(tmp_path):
    if shutil.which("g++") is None or not os.path.isdir(CUDA_INC):
        pytest.skip("needs g++ and the CUDA headers (vector types)")
    exe = tmp_path / "check_cache"
    cmd = ["g++", "-std=c++17", "-O2", "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-I", CUDA_INC,
           os.path.join(ROOT, "tests", "host", "check_cache.cpp"), os.path.join(CSRC, "cell_plan.cpp"),
           os.path.join(CSRC, "bvh_build.cpp"), "-o", str(exe), "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
