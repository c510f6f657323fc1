"""The serving arena (csrc/mtb_arena.h) on the host: first fit, complete
merging and the bound of holders + 1 free blocks, checked step by step against
a brute-force unit map over random alloc/release sequences (arena_check.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2007_06483_gb300", "csrc")


@pytest.fixture(scope="module")
def arena_check(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "arena_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6, 7, 8])
def test_arena_matches_first_fit_model(arena_check, seed):
    r = subprocess.run([arena_check, str(seed), "20000"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
