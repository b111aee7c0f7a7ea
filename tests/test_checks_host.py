"""Host check of the index predicates that a checked build
(DGW_DEVICE_CHECKS, libdgwave_checked.so) evaluates on the device before
each access it guards: face connection codes and block-table entries.  The
predicates are constexpr; this test compiles a C++ file of static_asserts
against them (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = r"""
#include "launch.h"
using dgw::block_ok;
using dgw::nbr_code_ok;
constexpr int code(int k, int f, int rev) { return k * 8 + f * 2 + rev; }
// a field of 100 values holds 10 elements of Np = 10
static_assert(nbr_code_ok(-1, 100, 10), "boundary face");
static_assert(nbr_code_ok(code(0, 0, 0), 100, 10), "first element");
static_assert(nbr_code_ok(code(9, 2, 1), 100, 10), "last element, face 2, reversed");
static_assert(!nbr_code_ok(code(10, 0, 0), 100, 10), "one element past the field");
static_assert(!nbr_code_ok(code(1 << 20, 1, 0), 100, 10), "far past the field");
static_assert(!nbr_code_ok(code(3, 3, 0), 100, 10), "face 3 does not exist");
static_assert(!nbr_code_ok(code(3, 3, 1), 100, 10), "face 3, reversed");
// blocks of at most 40 elements in a field of 400 values, Np = 10
static_assert(block_ok(0, 40, 40, 400, 10), "whole field");
static_assert(block_ok(36, 4, 40, 400, 10), "ragged last block");
static_assert(!block_ok(1, 40, 40, 400, 10), "one element past the field");
static_assert(!block_ok(0, 0, 40, 400, 10), "empty block");
static_assert(!block_ok(0, 41, 40, 400, 10), "longer than a block");
static_assert(!block_ok(-4, 4, 40, 400, 10), "negative first element");
int main() { return 0; }
"""


def test_index_predicates(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "checks.cpp"
    src.write_text(CASES)
    cmd = [nvcc, "-x", "c++", "-std=c++17", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_1304_5546_gb300", "csrc"), "-c", str(src),
           "-o", str(tmp_path / "checks.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
