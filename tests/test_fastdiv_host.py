"""CPU check of the multiply-high division the tile kernels use to find a cell's row and plane
(FastDiv in csrc/fresco_internal.h, the round-up method of Granlund and Montgomery): its host
path, which also computes the constants the plans hand to the device, against integer division,
exhaustively over small divisors and numerators and at the ends of the range. The device path
evaluates the same expression with __umulhi."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2305_15693_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "fresco_internal.h"
int main() {
    long bad = 0, checked = 0;
    unsigned long long s = 88172645463325252ULL;
    for (int d = 1; d <= 70000; d = d < 3000 ? d + 1 : d + 61) {
        const fresco::FastDiv f(d);
        const int nmax = d < 3000 ? 1 << 18 : 1 << 12;
        for (int n = 0; n < nmax; ++n, ++checked)
            if (f.div(n) != n / d) ++bad;
        for (int k = 0; k < 256; ++k, ++checked) {
            s ^= s << 13; s ^= s >> 7; s ^= s << 17;
            const int n = (int)(s & 0x7fffffffULL);
            if (f.div(n) != n / d) ++bad;
        }
        const int top = 0x7fffffff;
        ++checked;
        if (f.div(top) != top / d) ++bad;
    }
    std::printf("%ld %ld\n", bad, checked);
    return 0;
}
"""


def _cuda_include():
    for home in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if home and os.path.exists(os.path.join(home, "include", "cuda_runtime.h")):
            return os.path.join(home, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
        if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
            return inc
    return None


def test_fastdiv_matches_integer_division(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    src = tmp_path / "fastdiv.cpp"
    exe = tmp_path / "fastdiv"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                    "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    bad, checked = int(out[0]), int(out[1])
    assert checked > 700_000_000
    assert bad == 0
