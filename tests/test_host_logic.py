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


# (id, snippet of host_logic.h, replacement): each must make the check fail
MUTATIONS = [
    ("radix-2-before-4", "const int pref[] = {4, 2, 3, 5, 7};", "const int pref[] = {2, 4, 3, 5, 7};"),
    ("interleave-shifted", "per[k % grid].push_back", "per[(k + 1) % grid].push_back"),
    ("most-loaded-first", "std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;",
     "std::priority_queue<Load, std::vector<Load>, std::less<Load>> pq;"),
    ("lists-unsorted", "for (auto& v : per) std::sort(v.begin(), v.end());", "(void)per;"),
    ("bad-row-reported-late", "*bad_j = j;", "*bad_j = j + 1;"),
    ("row-offset-off-by-one", "rowoff[t + 1] = (int)rows.size();", "rowoff[t + 1] = (int)rows.size() + (t > 0);"),
]


@pytest.mark.parametrize("mid,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_check_catches_planted_slip(tmp_path, mid, old, new):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    hdr = os.path.join(ROOT, "paper_1203_4587_gb300", "csrc", "host_logic.h")
    with open(hdr) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"snippet not found exactly once: {old!r}"
    (tmp_path / "host_logic.h").write_text(src.replace(old, new))
    exe = tmp_path / "check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", str(tmp_path), os.path.join(ROOT, "tests", "host_logic_check.cpp"),
                    "-o", str(exe)], check=True, capture_output=True, text=True, timeout=120)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "FAIL" in r.stdout, f"{mid}: not caught"
