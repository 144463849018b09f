"""The invariant-divisor division the kernels use for line -> cell indices
(FastDivU32 / make_fastdiv in csrc/vk_kernels.h): the host-side multiplier and shifts,
applied with the kernels' formula (multiply-high, subtract, add, two shifts), must give
floor(n / d) for every 32-bit n.  Checked on the CPU with the header compiled by g++:
all divisors up to 4096 and the grid's actual ones (2304, 110592, ...) against edge
numerators (0, multiples of d and their neighbours, 2^31 +- 1, 2^32 - 1) and random ones.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2110_15867_gb300", "csrc")

SRC = r"""
#include "vk_kernels.h"
#include <cstdio>
#include <cstdint>
static unsigned apply(unsigned n, const vk::FastDivU32 &f)
{
    const unsigned t = unsigned((uint64_t(n) * f.m) >> 32);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}
int main()
{
    uint64_t x = 88172645463325252ull, bad = 0, checked = 0;
    auto rnd = [&]() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return unsigned(x); };
    const unsigned extra[] = {2304u, 3072u, 110592u, 147456u, 262144u, 884736u, 65535u, 65537u,
                              1000003u, 2147483647u, 2147483648u, 4294967295u};
    auto check = [&](unsigned d) {
        const vk::FastDivU32 f = vk::make_fastdiv(d);
        auto one = [&](unsigned n) {
            ++checked;
            if (apply(n, f) != n / d) {
                if (bad < 5) std::printf("d %u n %u: %u != %u\n", d, n, apply(n, f), n / d);
                ++bad;
            }
        };
        const unsigned edge[] = {0u, 1u, d - 1, d, d + 1, 2147483647u, 2147483648u, 2147483649u, 4294967295u,
                                 4294967294u};
        for (unsigned n : edge) one(n);
        for (unsigned k = 1; k < 64; ++k) {
            const uint64_t q = uint64_t(k) * d;
            if (q <= 4294967295ull) { one(unsigned(q)); one(unsigned(q - 1)); }
            const uint64_t top = (4294967295ull / d - k) * d;
            if (4294967295ull / d >= k) { one(unsigned(top)); one(unsigned(top - 1 + (top == 0))); }
        }
        for (int i = 0; i < 2000; ++i) one(rnd());
    };
    for (unsigned d = 1; d <= 4096; ++d) check(d);
    for (unsigned d : extra) check(d);
    for (int i = 0; i < 2000; ++i) check(rnd() | 1u);
    std::printf("checked %llu bad %llu\n", (unsigned long long)checked, (unsigned long long)bad);
    return bad != 0;
}
"""


def test_fastdiv_matches_integer_division(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    cuda_inc = None
    for cand in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda.h")):
            cuda_inc = os.path.join(cand, "include")
            break
    if cuda_inc is None:
        pytest.skip("CUDA headers not found")
    src = tmp_path / "fastdiv.cpp"
    exe = tmp_path / "fastdiv"
    src.write_text(SRC)
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    print(out.stdout)
    assert out.returncode == 0, out.stdout
