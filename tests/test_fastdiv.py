"""Host check of the multiply-shift division the lattice kernels use for site
coordinates (csrc/plq_fastdiv.h, compiled here by the host compiler): for every
divisor up to 4096 and every dividend in [0, 2^20), plus dividends near 2^31 and
random ones, the quotient and remainder equal integer division's."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include <initializer_list>
#include "plq_fastdiv.h"
int main() {
    uint64_t state = 0x9E3779B97F4A7C15ull, checked = 0;
    for (uint32_t d = 1; d <= 4096; ++d) {
        const plq::FastDiv f = plq::make_fastdiv(d);
        auto check = [&](uint32_t n) {
            uint32_t r = 0;
            const uint32_t q = plq::fd_divmod(n, f, &r);
            ++checked;
            if (q != n / d || r != n % d) {
                std::printf("FAIL d=%u n=%u q=%u r=%u\n", d, n, q, r);
                return false;
            }
            return true;
        };
        for (uint32_t n = 0; n < (1u << 20); n += (d < 64 ? 1 : 7)) if (!check(n)) return 1;
        for (uint32_t n = 0x7fffffffu - 4096; n < 0x7fffffffu; ++n) if (!check(n)) return 1;
        for (int k = 0; k < 2000; ++k) {
            state ^= state << 13; state ^= state >> 7; state ^= state << 17;
            if (!check((uint32_t)(state & 0x7fffffffu))) return 1;
        }
    }
    const uint32_t big[] = {65535u, 65536u, 1u << 20, 1000003u, 1u << 30, 0x7fffffffu};
    for (uint32_t d : big) {
        const plq::FastDiv f = plq::make_fastdiv(d);
        for (uint32_t n : {0u, d - 1, d, d + 1, 2 * d - 1, 0x7fffffffu, 0x7ffffffeu}) {
            if (n > 0x7fffffffu) continue;
            uint32_t r = 0;
            const uint32_t q = plq::fd_divmod(n, f, &r);
            if (q != n / d || r != n % d) { std::printf("FAIL d=%u n=%u\n", d, n); return 1; }
        }
    }
    std::printf("ok %llu\n", (unsigned long long)checked);
    return 0;
}
"""


def test_fast_division_matches_integer_division(tmp_path):
    src = tmp_path / "fastdiv_check.cpp"
    exe = tmp_path / "fastdiv_check"
    src.write_text(PROGRAM)
    inc = os.path.join(ROOT, "paper_1405_0700_gb300", "csrc")
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I" + inc, str(src), "-o", str(exe)], capture_output=True,
                       text=True)
    if r.returncode != 0:
        pytest.fail(r.stderr)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
