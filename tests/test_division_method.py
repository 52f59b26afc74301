"""Markstein's division by a small integer (the screened kernel's centroid
division): q0 = s*y, r = fma(-q0, N, s), q = fma(r, y, q0) with y = RN(1/N)
must equal the IEEE quotient s/N.  Checked on the host's IEEE arithmetic
(libm fma is correctly rounded) over random and structured operands; the GPU
parity tests then check the device results against the oracle."""
import os
import subprocess
import tempfile

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t next(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }
static double from_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
int main(int argc, char **argv) {
    long per = atol(argv[1]);
    long bad = 0, tested = 0;
    for (int N = 1; N <= 16; ++N) {
        double y = 1.0 / (double)N, fN = (double)N;
        for (long k = 0; k < per; ++k) {
            uint64_t r = next();
            double s;
            if (k % 4 == 0) s = from_bits((r & 0x800FFFFFFFFFFFFFull) | ((uint64_t)(1023 + (int)(r >> 52) % 64 - 32) << 52));
            else if (k % 4 == 1) s = (double)(int64_t)(r >> 11) * 0x1p-50;          /* multiples of a unit */
            else if (k % 4 == 2) s = (double)N * from_bits(0x3FF0000000000000ull | (r & 0xFFFFFFFFFFFFFull)) + (double)((int64_t)(r >> 60) - 8) * 0x1p-52;
            else s = from_bits((r & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull) * (double)N;
            double q0 = s * y;
            double rr = fma(-q0, fN, s);
            double q = fma(rr, y, q0);
            double ref = s / fN;
            if (memcmp(&q, &ref, 8) != 0) { if (bad < 5) printf("N=%d s=%a got %a want %a\n", N, s, q, ref); ++bad; }
            ++tested;
        }
    }
    printf("tested %ld bad %ld\n", tested, bad);
    return bad != 0;
}
"""


def test_markstein_small_integer_division_is_correctly_rounded():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "m.c")
        exe = os.path.join(d, "m")
        open(src, "w").write(SRC.replace("#include <string.h>", "#include <string.h>\n#include <stdlib.h>"))
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", src, "-o", exe, "-lm"], check=True)
        r = subprocess.run([exe, "2000000"], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
        assert "bad 0" in r.stdout
