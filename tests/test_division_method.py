"""The screened kernel's centroid division (csrc/div_small.cuh): q0 = RN(s*y)
with y = RN(1/N), then an exact integer remainder picks the correctly
rounded quotient.  It must equal the IEEE quotient s/N bit for bit.  The
header compiles for the host, so this runs the kernel's own code against the
host's IEEE division over random and structured operands: significands at the
bottom and top of a binade, exact multiples of N, odd multiples of N/2, both
signs, quotients next to a power of two, and exponents at the edges of the
fast path."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1502_00355_gb300", "csrc")

SRC = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "div_small.cuh"
using namespace sls::divs;
static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t nxt(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }
int main(int argc, char **argv) {
    long per = atol(argv[1]);
    long bad = 0, tested = 0, fast = 0;
    for (uint32_t N = 2; N <= 16; ++N) {
        const double y = 1.0 / (double)N, fN = (double)N;
        for (long k = 0; k < per; ++k) {
            uint64_t r = nxt(), r2 = nxt();
            uint64_t sign = (r2 & 1) ? 0x8000000000000000ull : 0ull;
            int e = 1023 + (int)(r2 >> 40) % 200 - 100;
            uint64_t mant;
            switch (k % 9) {
            case 0: mant = r & 0x000FFFFFFFFFFFFFull; break;                       /* random */
            case 1: mant = (r & 0xFFull); break;                                   /* bottom of a binade */
            case 2: mant = 0x000FFFFFFFFFFFFFull - (r & 0xFFull); break;           /* top of a binade */
            case 3: mant = r & 0x000FFFFFFFFFF000ull; break;                       /* short significands */
            case 4: { double v = (double)N * (double)((r >> 12) | 1ull);            /* exact multiples of N */
                      uint64_t b = bits_of(v); mant = b & 0x000FFFFFFFFFFFFFull; break; }
            case 5: { double v = (double)N * ((double)(r >> 11) + 0.5);             /* halfway quotients */
                      uint64_t b = bits_of(v); mant = b & 0x000FFFFFFFFFFFFFull; break; }
            case 6: mant = r & 0x000FFFFFFFFFFFFFull; e = (k & 16) ? 63 + (int)(r2 % 8) : 2000 - (int)(r2 % 8); break;
            case 7: { /* within a few units of N * 2^j: quotients at the edges of a binade */
                      uint64_t b = bits_of((double)N * (double)(1ull << (r2 % 40))) + (r % 9) - 4;
                      e = (int)((b >> 52) & 0x7ff); mant = b & 0x000FFFFFFFFFFFFFull; break; }
            default: mant = r & 0x000FFFFFFFFFFFFFull; e = 1 + (int)(r2 % 2046); break;   /* any exponent */
            }
            uint64_t sb = sign | ((uint64_t)e << 52) | mant;
            uint64_t got = div_small_bits(sb, N, y, fN);
            double want = of_bits(sb) / fN;
            if (got != bits_of(want)) {
                if (bad < 8) printf("N=%u s=%a got %a want %a\n", N, of_bits(sb), of_bits(got), want);
                ++bad;
            }
            ++tested;
            fast += (e >= 63 && e <= 2000);
        }
    }
    printf("tested %ld fast %ld bad %ld\n", tested, fast, bad);
    return bad != 0;
}
"""


def test_small_integer_division_is_correctly_rounded():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "m.cpp")
        exe = os.path.join(d, "m")
        open(src, "w").write(SRC)
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, src, "-o", exe], check=True)
        r = subprocess.run([exe, "2000000"], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout
        assert "bad 0" in r.stdout
