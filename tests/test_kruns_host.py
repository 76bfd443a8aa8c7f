"""Host logic of the sigma tasks' K runs (no GPU): compiles tests/kruns_check.cpp
against the library's kruns.hpp with the host C++ compiler and runs its
randomised checks.  Every non-zero column must be read by exactly one run,
runs start on 8-column boundaries (16-byte TMA coordinates), and the exact
merge of the FP64 path is the union of the ranges."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1509_00216_gb300", "csrc")


def test_k_runs_read_every_nonzero_column_exactly_once(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "kruns_check")
    build = subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "kruns_check.cpp"), "-o", exe],
                           capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert run.stdout.strip().endswith("ok")
