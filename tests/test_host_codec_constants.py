"""Host logic of the fixed-point storage: the codec constants qscale_of_exponent
(csrc/lbm_internal.h) builds, with and without a reference shift.  A C++ program compiled
against the header applies them with IEEE fused multiply-adds (the operation the kernels issue)
and checks, for grid steps 2^e from 2^-23 to 2^-7 and shifts of up to 2^22 grid steps:
- every constant is exactly representable (no rounding of the shift into the constants);
- encoding h gives the nearest code, round(h / 2^e - k + 2^15) with ties to an even code (the
  storage type's own rounding; with no shift, k = 0, that is ties to an even grid point), and
  decoding that code gives its grid point, (code - 2^15 + k) 2^e, exactly;
- the range check (the upper half of the encoded bits changes) fires exactly when the unrounded
  code c = h / 2^e - k + 2^15 lies outside [-1/4, 2^16 - 1/2): above, c rounds to 2^16 or more;
  below, the fused sum 2^23 + c falls under 2^23, where FP32 steps by 1/2, so the last quarter
  step before code 0 still rounds into it and anything lower is flagged.
The kernels' own encode and decode are checked against these rules on the GPU
(tests/test_gpu_fixed_point.py); this pins the constants on the host.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = "/usr/local/cuda"

PROGRAM = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include "lbm_internal.h"

static uint64_t x = 0x2545F4914F6CDD1Dull;
static uint64_t rnd() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; }  // xorshift64
static double uni() { return (rnd() >> 11) * (1.0 / 9007199254740992.0); }

static unsigned int bits(float f) { unsigned int b; memcpy(&b, &f, 4); return b; }
static float flt(unsigned int b) { float f; memcpy(&f, &b, 4); return f; }

int main() {
    const int Q = 39;
    int bad = 0;
    for (int e = -23; e <= -7 && !bad; ++e) {
        const double step = ldexp(1.0, e);
        for (int trial = 0; trial < 200 && !bad; ++trial) {
            double ref[Q];
            for (int i = 0; i < Q; ++i) ref[i] = (uni() * 2.0 - 1.0) * ldexp(1.0, 22) * step * (trial % 2 ? 1.0 : 1e-3);
            const lbm::QScale q = trial % 5 == 0 ? lbm::qscale_of_exponent(e) : lbm::qscale_of_exponent(e, ref, Q);
            const bool shifted = trial % 5 != 0;
            for (int i = 0; i < Q && !bad; ++i) {
                const double k = shifted ? rint(ref[i] / step) : 0.0;
                if ((double)q.enc[i] != 8421376.0 - k || (double)q.dec[i] != -(8421376.0 - k) * step ||
                    (double)q.mul != step || (double)q.inv != 1.0 / step) {
                    printf("e=%d i=%d: constants not exact\n", e, i);
                    bad = 1;
                    break;
                }
                for (int s = 0; s < 64; ++s) {
                    // h within a few steps of the range around the shift, on or between grid
                    // points, ties and both ends included
                    double code = floor(uni() * 65536.0);
                    if (s % 8 == 3) code = -1.0 - floor(uni() * 3.0);
                    if (s % 8 == 7) code = 65535.0 + floor(uni() * 3.0);
                    double g = code - 32768.0 + k;               // grid units
                    if (s % 4 == 1) g += 0.5;                        // a tie
                    else if (s % 4 == 2) g += uni() - 0.5;           // anywhere
                    const float h = (float)(g * step);
                    const double hg = (double)h / step;             // h in grid units, exact
                    const double c = hg - k + 32768.0;                 // unrounded code, exact
                    const double wcode = nearbyint(c);                 // ties to an even code
                    const double want = wcode - 32768.0 + k;           // its grid point
                    const unsigned int v = bits(fmaf(h, q.inv, q.enc[i]));
                    const bool inside = c >= -0.25 && c < 65535.5;
                    if (((v ^ 0x4B000000u) >> 16 != 0u) == inside) {
                        printf("e=%d i=%d h=%.17g: range check wrong\n", e, i, (double)h);
                        bad = 1;
                        break;
                    }
                    if (!inside) continue;
                    if ((v & 0xFFFFu) != (unsigned int)wcode) {
                        printf("e=%d i=%d h=%.17g: code %u want %.0f\n", e, i, (double)h, v & 0xFFFFu, wcode);
                        bad = 1;
                        break;
                    }
                    const float d = fmaf(flt(0x4B000000u | (v & 0xFFFFu)), q.mul, q.dec[i]);
                    if ((double)d != want * step) {
                        printf("e=%d i=%d: decode %.17g want %.17g\n", e, i, (double)d, want * step);
                        bad = 1;
                        break;
                    }
                }
            }
        }
        // beyond the range: one grid step past either end is flagged
        const lbm::QScale q = lbm::qscale_of_exponent(e);
        const float lo = (float)(-32769.0 * step), hi = (float)(32768.0 * step);
        if ((bits(fmaf(lo, q.inv, q.enc[0])) ^ 0x4B000000u) >> 16 == 0u ||
            (bits(fmaf(hi, q.inv, q.enc[0])) ^ 0x4B000000u) >> 16 == 0u) {
            printf("e=%d: ends of the range not flagged\n", e);
            bad = 1;
        }
    }
    if (!bad) printf("ok\n");
    return bad;
}
"""


def test_fixed_point_codec_constants(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("g++ or the CUDA headers not found")
    src = tmp_path / "codec.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "codec"
    # -ffp-contract=off: the program's own arithmetic stays as written; fmaf is the fused operation
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I",
                        os.path.join(ROOT, "paper_2002_02503_gb300", "csrc"), "-I", os.path.join(CUDA, "include"),
                        str(src), "-o", str(exe), "-lm"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
