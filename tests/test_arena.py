"""The device-memory sub-allocator's host logic, compiled with g++ and run
with random allocate/release sequences (no GPU; see tests/native/arena_stress.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.parametrize("seed", [1, 2])
def test_arena_stress(tmp_path, seed):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    exe = tmp_path / "arena_stress"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2509_08383_gb300", "csrc"),
                    os.path.join(HERE, "native", "arena_stress.cpp"), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe), str(seed)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok")
