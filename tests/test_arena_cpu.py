"""Host-only check of the serving arena's sub-allocator (csrc/arena.h):
compiled with g++ and run on randomised alloc/free sequences against a
unit-by-unit model."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "native", "arena_check.cpp")
INC = os.path.join(ROOT, "paper_2308_07932_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if not shutil.which("g++"):
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", INC, SRC, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_arena_against_model(checker, seed):
    out = subprocess.run([checker, str(seed), "6000"], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
