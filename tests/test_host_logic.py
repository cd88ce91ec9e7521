"""The library's host-side planning logic on the CPU: FFT stage radices for
every transform length and the per-CTA column work lists of batched solves
(paper_1203_4587_gb300/csrc/host_logic.h), checked by a small C++ program
built with the host compiler."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_planning_logic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "host_logic_check"
    src = os.path.join(ROOT, "tests", "host_logic_check.cpp")
    inc = os.path.join(ROOT, "paper_1203_4587_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", inc, src, "-o", str(exe)], check=True,
                   capture_output=True, text=True, timeout=120)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-2000:]
