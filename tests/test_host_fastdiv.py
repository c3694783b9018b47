"""Host logic of the batched step: the constants fastdiv_init (csrc/lbm_internal.h) computes for
the batch kernels' division by a runtime divisor.  A small C++ program compiled against the
header checks q = (umulhi(n, m) + n) >> s, the form the kernels evaluate, against n / d for every
divisor up to 4096 (the lattice widths and row counts a pool meets) and for random divisors up to
2^31 - 1, with numerators at both ends of [0, 2^31) and between.  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = "/usr/local/cuda"

PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include "lbm_internal.h"

static unsigned int q_of(unsigned int n, unsigned int m, unsigned int s) {
    const unsigned int hi = (unsigned int)(((uint64_t)n * m) >> 32);  // umulhi
    return (hi + n) >> s;
}

static int check(unsigned int d, unsigned int n) {
    unsigned int m, s;
    lbm::fastdiv_init(d, &m, &s);
    if (q_of(n, m, s) != n / d) {
        printf("d=%u n=%u got %u want %u\n", d, n, q_of(n, m, s), n / d);
        return 1;
    }
    return 0;
}

int main() {
    uint64_t x = 88172645463325252ull;  // xorshift64 (Marsaglia 2003)
    int bad = 0;
    for (unsigned int d = 1; d <= 4096 && !bad; ++d) {
        for (unsigned int n = 0; n < 3 * d + 2 && !bad; ++n) bad |= check(d, n);  // near multiples
        const unsigned int top = 0x7fffffffu;
        for (unsigned int k = 0; k < 64 && !bad; ++k) bad |= check(d, top - k);
        for (unsigned int k = 0; k < 64 && !bad; ++k) bad |= check(d, (top / d) * d - k % 2);
        for (int r = 0; r < 256 && !bad; ++r) {
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            bad |= check(d, (unsigned int)(x & 0x7fffffffu));
        }
    }
    for (int r = 0; r < 200000 && !bad; ++r) {
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        const unsigned int d = (unsigned int)((x >> 33) & 0x7fffffffu) | 1u;
        x ^= x << 13; x ^= x >> 7; x ^= x << 17;
        bad |= check(d, (unsigned int)(x & 0x7fffffffu));
        bad |= check(d, d - 1) | check(d, d) | check(d, 0x7fffffffu);
    }
    if (!bad) printf("ok\n");
    return bad;
}
"""


def test_fastdiv_constants_divide_exactly(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("g++ or the CUDA headers not found")
    src = tmp_path / "fastdiv.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "fastdiv"
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2002_02503_gb300", "csrc"),
                        "-I", os.path.join(CUDA, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
