"""Host logic: the invariant-divisor division that the grid-stride kernels use
to split a flat index into (sample, row, column) agrees with integer division
for the level sides, their squares and products of the workloads, powers of
two, odd divisors and the extremes (fastdiv_check.cpp, built with g++)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fastdiv_matches_integer_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = tmp_path / "fastdiv_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1806_05619_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fastdiv_check.cpp"), "-o", str(exe)], check=True)
    sides = [8 << t for t in range(9)] + [12, 24, 48, 96, 160]
    divisors = set(sides)
    divisors |= {n * n for n in sides} | {(n // 2) ** 2 for n in sides} | {n * (n // 2) for n in sides}
    divisors |= {n * (n // 4) for n in sides} | {n * ka for n in sides for ka in (1, 7, 32, 100)}
    divisors |= {1, 2, 3, 5, 7, 641, 65535, 65536, 65537, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 1}
    out = subprocess.run([str(exe)] + [str(d) for d in sorted(divisors)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
