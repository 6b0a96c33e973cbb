"""The sweep's division by a Block's width and height (div_magic / quot in
csrc/sweep_types.h, the multiply-shift method of Granlund and Montgomery)
against plain integer division, compiled with the host compiler: every
divisor up to 4096 with quotients 0..1000 at both ends of each remainder
range, larger divisors up to 2^30, and dividends up to 2^31 - 1."""
import os
import shutil
import subprocess

import pytest

from paper_1007_1388_gb300 import build

SRC = r"""
#include "sweep_types.h"
#include <cstdint>
#include <cstdio>
#include <random>

static long long n_tests = 0, n_bad = 0;

static void check(uint32_t d, uint32_t m, int sh, uint64_t n)
{
    if (n >= (1ull << 31)) return;
    ++n_tests;
    if (lbm::quot(int(n), m, sh) != int(n / d)) {
        if (n_bad < 5) std::printf("d=%u n=%llu\n", d, (unsigned long long)n);
        ++n_bad;
    }
}

int main()
{
    std::mt19937_64 rng(7);
    for (uint64_t d = 1; d <= (1ull << 30); d = d < 4096 ? d + 1 : d * 3 + 1) {
        uint32_t m;
        int sh;
        lbm::div_magic(uint32_t(d), &m, &sh);
        for (uint64_t k = 0; k <= 1000; ++k) {
            check(uint32_t(d), m, sh, k * d);
            check(uint32_t(d), m, sh, k * d + d - 1);
        }
        const uint64_t top = (1ull << 31) - 1;
        check(uint32_t(d), m, sh, top);
        check(uint32_t(d), m, sh, top - top % d);
        if (top % d) check(uint32_t(d), m, sh, top - top % d - 1);
        for (int r = 0; r < 64; ++r) check(uint32_t(d), m, sh, rng() & 0x7fffffffull);
    }
    std::printf("%lld %lld\n", n_tests, n_bad);
    return n_bad != 0;
}
"""


def test_quot_equals_integer_division(tmp_path):
    cxx = shutil.which("g++")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if cxx is None or not os.path.exists(os.path.join(cuda, "include", "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "quot.cpp"
    src.write_text(SRC)
    exe = tmp_path / "quot"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + os.path.join(cuda, "include"), "-I" + build.CSRC,
                    "-I" + os.path.join(build.ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    tests, bad = (int(v) for v in out.stdout.split()[-2:])
    assert out.returncode == 0 and bad == 0, out.stdout
    assert tests > 8_000_000
