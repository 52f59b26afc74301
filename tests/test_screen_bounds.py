"""The FP32 screen of the accept test (csrc/screen.cuh), checked on the CPU.

The screened kernel is bit-exact only if, for every incident triangle, the
FP64 alpha that the exact definition computes lies inside the interval
[a - b, a + b] around the screen's FP32 alpha a, and if the difference screen
never claims a sign that the FP64 comparison of q_new and q_old does not
have.  The header compiles for the host, so this runs the kernel's own code
(head/tail splits, the local frame, screen_alpha, side_g, side_bound,
bound_ok, frame_ok, diff_screen and the constants kC1..kC3, kGMax, kE64,
kLocalRange) on adversarial triangles and compares it with

* alpha in binary128 (K * cross / s from the FP64 inputs, K the double
  nearest 2 sqrt(3)): |a - alpha| <= b;
* alpha in the FP64 expression tree of the definition (what the oracle
  computes): |a - alpha_fp64| <= b;
* the sign of alpha_fp64(centre) - alpha_fp64(node) wherever diff_screen
  returns +-1.

The device's approximate reciprocal is within 2 ulp of 1/s; the host stand-in
is shifted by -2, 0 and +2 ulp in three runs.  Families of triangles: well
shaped, slivers, equilateral and inverted equilateral (|alpha| near 1),
centres moved next to two far neighbours (g = R^2/s up to kGMax and past it),
rings at the 2^-20 M limit of the local frame, coordinates straddling a power
of two or zero, and moves of a few ulps up to 1e-3 of the ring.  A test that
weakens a constant (plants a smaller bound in a copy of the header) must
fail, which shows the families reach the bounds.
"""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1502_00355_gb300", "csrc")

HARNESS = r"""
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
static int g_rcp_shift = 0;
static float host_rcp(float s) {
    float r = 1.0f / s;
    for (int k = 0; k < g_rcp_shift; ++k) r = nextafterf(r, INFINITY);
    for (int k = 0; k > g_rcp_shift; --k) r = nextafterf(r, -INFINITY);
    return r;
}
#define SLS_SCREEN_HOST_RCP(s) host_rcp(s)
#include "screen.cuh"
using namespace sls::scr;

#if defined(__x86_64__) || defined(__i386__)
typedef __float128 qreal;
#else
typedef long double qreal; /* binary128 on aarch64 Linux */
#endif

static const double kK = 3.4641016151377544;
static uint64_t st = 0x2545F4914F6CDD1Dull;
static uint64_t nxt(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }
static double u01(void) { return (double)(nxt() >> 11) * (1.0 / 9007199254740992.0); }
static double uni(double a, double b) { return a + (b - a) * u01(); }
static uint64_t bits(double v) { uint64_t b; memcpy(&b, &v, 8); return b; }

struct P { double x, y; };

/* alpha of (a, b, c) in stored order, FP64 tree of the definition */
static double alpha64(P a, P b, P c) {
    double e1x = b.x - a.x, e1y = b.y - a.y, e2x = c.x - a.x, e2y = c.y - a.y, e3x = c.x - b.x, e3y = c.y - b.y;
    double cr = e1x * e2y - e1y * e2x;
    double l1 = e1x * e1x + e1y * e1y, l2 = e2x * e2x + e2y * e2y, l3 = e3x * e3x + e3y * e3y;
    double s = (l1 + l2) + l3;
    return s > 0.0 ? (kK * cr) / s : 0.0;
}
static qreal alphaq(P a, P b, P c) {
    qreal e1x = (qreal)b.x - a.x, e1y = (qreal)b.y - a.y, e2x = (qreal)c.x - a.x, e2y = (qreal)c.y - a.y;
    qreal e3x = (qreal)c.x - b.x, e3y = (qreal)c.y - b.y;
    qreal cr = e1x * e2y - e1y * e2x;
    qreal s = (e1x * e1x + e1y * e1y) + (e2x * e2x + e2y * e2y) + (e3x * e3x + e3y * e3y);
    return s > 0 ? ((qreal)kK * cr) / s : (qreal)0;
}
static P stored(int slot, int k, P node, P A, P B) {
    /* k-th vertex of the stored triangle whose node slot is `slot`, A, B the others in order */
    P v[3];
    int j = 0;
    for (int t = 0; t < 3; ++t) v[t] = (t == slot) ? node : (j++ == 0 ? A : B);
    return v[k];
}

static long n_tri = 0, n_checked = 0, n_bad = 0, n_diff = 0, n_diff_checked = 0;
static long n_frame_fail = 0, n_bound_fail = 0;
static double worst_q = 0.0, worst_64 = 0.0;

static void check(int fam, P p, P A, P B, P c, int slot, double rho) {
    ++n_tri;
    float phx, plx, phy, ply;
    bool ok = head_tail(bits(p.x), phx, plx) & head_tail(bits(p.y), phy, ply);
    float Ax, Ay, Bx, By;
    bool oka, okb;
    local_offset(bits(A.x), bits(A.y), phx, plx, phy, ply, Ax, Ay, oka);
    local_offset(bits(B.x), bits(B.y), phx, plx, phy, ply, Bx, By, okb);
    ok = ok & oka & okb;
    const float rlA = fmaxf(fabsf(Ax), fabsf(Ay)), rlB = fmaxf(fabsf(Bx), fabsf(By));
    /* other neighbours of the node may reach further: rn >= this triangle's */
    const float rn = fmaxf(fmaxf(rlA, rlB), (float)rho);
    const float rmin = fminf(rlA, rlB);
    const double dx = c.x - p.x, dy = c.y - p.y;
    const float Cx = trunc_float(bits(dx)), Cy = trunc_float(bits(dy));
    const float rC = fmaxf(fabsf(Cx), fabsf(Cy));
    const float M = fmaxf(fabsf(phx), fabsf(phy)) * 1.0001f + fmaxf(rn, rC);
    if (!ok || !frame_ok(rmin, fmaxf(rn, rC), M)) { ++n_frame_fail; return; }
    const float sk = slot == 1 ? -kTwoSqrt3f : kTwoSqrt3f;
    const float ba2 = edge_ba2(Ax, Ay, Bx, By);
    for (int side = 0; side < 2; ++side) {
        float sv;
        const float X0 = side ? Cx : 0.0f, X1 = side ? Cy : 0.0f;
        const float a = screen_alpha(X0, X1, Ax, Ay, Bx, By, ba2, sk, sv);
        const float R = side ? fmaxf(rn, rC) : rn;
        const float g = side_g(R, sv);
        const float amax = fabsf(a);
        if (!bound_ok(sv, g, amax)) { ++n_bound_fail; continue; }
        const float b = side_bound(amax, g);
        const P node = side ? c : p;
        const P t0 = stored(slot, 0, node, A, B), t1 = stored(slot, 1, node, A, B), t2 = stored(slot, 2, node, A, B);
        const double a64 = alpha64(t0, t1, t2);
        const qreal aq = alphaq(t0, t1, t2);
        double eq = (double)((qreal)a - aq);
        eq = eq < 0 ? -eq : eq;
        double e64 = fabs((double)a - a64);
        ++n_checked;
        if (eq / b > worst_q) worst_q = eq / b;
        if (e64 / b > worst_64) worst_64 = e64 / b;
        if (!(eq <= (double)b) || !(e64 <= (double)b)) {
            if (n_bad < 10)
                printf("BAD fam %d side %d slot %d a %.9g exact %.17g fp64 %.17g bound %.3g g %.3g\n", fam, side, slot,
                       (double)a, (double)aq, a64, (double)b, (double)g);
            ++n_bad;
        }
    }
    /* the difference screen: the sign it claims must be that of q_new - q_old */
    const int v = diff_screen(Ax, Ay, Bx, By, Cx, Cy, slot == 1 ? -1.0f : 1.0f, M * M);
    ++n_diff_checked;
    if (v != 0) {
        ++n_diff;
        const P o0 = stored(slot, 0, p, A, B), o1 = stored(slot, 1, p, A, B), o2 = stored(slot, 2, p, A, B);
        const P m0 = stored(slot, 0, c, A, B), m1 = stored(slot, 1, c, A, B), m2 = stored(slot, 2, c, A, B);
        const double qo = alpha64(o0, o1, o2), qn = alpha64(m0, m1, m2);
        const qreal d = alphaq(m0, m1, m2) - alphaq(o0, o1, o2);
        const int s64 = qn > qo ? 1 : (qn < qo ? -1 : 0);
        const int sq = d > 0 ? 1 : (d < 0 ? -1 : 0);
        if (s64 != v || sq != v) {
            if (n_bad < 10) printf("BAD diff fam %d v %d fp64 %d exact %d qo %.17g qn %.17g\n", fam, v, s64, sq, qo, qn);
            ++n_bad;
        }
    }
}

static P rot(double r, double th) { P q = {r * cos(th), r * sin(th)}; return q; }
static P add(P a, P b) { P q = {a.x + b.x, a.y + b.y}; return q; }

int main(int argc, char **argv) {
    const long per = atol(argv[1]);
    g_rcp_shift = atoi(argv[2]);
    st ^= (uint64_t)(g_rcp_shift + 7) * 0x9E3779B97F4A7C15ull;
    for (long k = 0; k < per; ++k) {
        const int fam = (int)(k % 9);
        const int slot = (int)(nxt() % 3);
        P p = {uni(0.0, 1.0), uni(0.0, 1.0)};
        double h = ldexp(1.0, -(int)(5 + nxt() % 16));   /* ring size 2^-5 .. 2^-20 */
        double th = uni(0.0, 6.283185307179586);
        P A, B, c;
        double rho = 0.0;
        switch (fam) {
        case 0: /* well shaped, random move towards somewhere in the ring */
            A = add(p, rot(h * uni(0.5, 1.5), th));
            B = add(p, rot(h * uni(0.5, 1.5), th + uni(0.5, 2.5)));
            c = add(p, rot(h * uni(0.0, 0.7), uni(0.0, 6.3)));
            break;
        case 1: /* slivers: B nearly on the line p-A, or A and B nearly coincident */
            A = add(p, rot(h, th));
            if (nxt() & 1) B = add(p, rot(h * uni(0.2, 2.0), th + (nxt() & 1 ? 1 : -1) * ldexp(uni(1, 2), -(int)(4 + nxt() % 40))));
            else B = add(A, rot(h * ldexp(uni(1, 2), -(int)(3 + nxt() % 18)), uni(0, 6.3)));
            c = add(p, rot(h * uni(0.0, 0.5), uni(0.0, 6.3)));
            rho = (nxt() & 1) ? h * uni(1.0, 30.0) : 0.0;
            break;
        case 2: /* |alpha| near 1: equilateral, either orientation */
            A = add(p, rot(h, th));
            B = add(p, rot(h, th + ((nxt() & 1) ? 1.0471975511965976 : -1.0471975511965976) * uni(0.999, 1.001)));
            c = add(p, rot(h * ldexp(1.0, -(int)(nxt() % 30)), uni(0.0, 6.3)));
            break;
        case 3: { /* centre next to two far neighbours: g = R^2 / s large */
            A = add(p, rot(h, th));
            const double r = h * ldexp(uni(1, 2), -(int)(1 + nxt() % 7));
            B = add(A, rot(r, uni(0, 6.3)));
            c = add(A, rot(r * uni(0.3, 1.0), uni(0, 6.3)));
            break;
        }
        case 4: { /* ring at the 2^-20 M limit of the local frame */
            const double mag = ldexp(1.0, (int)(nxt() % 21) - 10);
            p.x = mag * uni(0.5, 1.0); p.y = mag * uni(-1.0, 1.0);
            const double M = fmax(fabs(p.x), fabs(p.y));
            h = M * ldexp(1.0, -20) * uni(1.0, 1.3);
            A = add(p, rot(h * uni(1.0, 1.5), th));
            B = add(p, rot(h * uni(1.0, 1.5), th + uni(0.8, 2.2)));
            c = add(p, rot(h * uni(0.0, 0.5), uni(0, 6.3)));
            break;
        }
        case 5: { /* straddling a power of two, or zero */
            const double pw = (nxt() & 1) ? ldexp(1.0, -(int)(nxt() % 12)) : 0.0;
            p.x = pw + h * uni(-0.3, 0.3); p.y = ((nxt() & 1) ? pw : 0.5) + h * uni(-0.3, 0.3);
            A = add(p, rot(h * uni(0.5, 1.5), th));
            B = add(p, rot(h * uni(0.5, 1.5), th + uni(0.5, 2.5)));
            c = add(p, rot(h * uni(0.0, 0.7), uni(0.0, 6.3)));
            if (nxt() & 1) { A.x = pw; }  /* a neighbour exactly on the power of two or on zero */
            break;
        }
        case 6: case 7: { /* moves of a few ulps of the node up to 1e-3 of the ring */
            A = add(p, rot(h * uni(0.5, 1.5), th));
            B = add(p, rot(h * uni(0.5, 1.5), th + uni(0.3, 2.8)));
            if (fam == 6) {
                c.x = nextafter(p.x, (nxt() & 1) ? 2.0 : -2.0);
                c.y = p.y;
                for (int q = (int)(nxt() % 64); q > 0; --q) c.y = nextafter(c.y, (nxt() & 1) ? 2.0 : -2.0);
            } else {
                c = add(p, rot(h * ldexp(1.0, -(int)(10 + nxt() % 33)), uni(0, 6.3)));
            }
            break;
        }
        default: { /* inverted or nearly degenerate triangles with large moves */
            A = add(p, rot(h, th));
            B = add(p, rot(h * uni(0.1, 1.0), th + uni(-0.2, 0.2)));
            c = add(p, rot(h * uni(0.5, 2.0), uni(0.0, 6.3)));
            break;
        }
        }
        check(fam, p, A, B, c, slot, rho);
    }
    printf("triangles %ld checked %ld frame_fail %ld bound_fail %ld diff_decided %ld/%ld worst_q %.4f worst_64 %.4f bad %ld\n",
           n_tri, n_checked, n_frame_fail, n_bound_fail, n_diff, n_diff_checked, worst_q, worst_64, n_bad);
    return n_bad != 0;
}
"""


def _build(d, header_dir):
    src = os.path.join(d, "h.cpp")
    exe = os.path.join(d, "h")
    with open(src, "w") as f:
        f.write(HARNESS)
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-I", header_dir,
                    src, "-o", exe, "-lm"], check=True)
    return exe


def _run(exe, per, shift):
    r = subprocess.run([exe, str(per), str(shift)], capture_output=True, text=True)
    return r.returncode, r.stdout


@pytest.mark.parametrize("shift", [-2, 0, 2])
def test_screen_alpha_bound_and_difference_screen(shift):
    with tempfile.TemporaryDirectory() as d:
        exe = _build(d, CSRC)
        rc, out = _run(exe, 450_000, shift)
        assert rc == 0, out
        m = re.search(r"triangles (\d+) checked (\d+) .* diff_decided (\d+)/(\d+) worst_q ([\d.]+) worst_64 ([\d.]+) bad (\d+)",
                      out)
        assert m, out
        tri, checked, decided = int(m.group(1)), int(m.group(2)), int(m.group(3))
        # two sides per triangle: at least 1e6 bound checks over the three runs' worth
        assert checked >= 500_000 and decided >= 50_000, out
        # the bounds hold with the margin the derivation leaves (factor 1.5)
        assert float(m.group(5)) < 1.0 and float(m.group(6)) < 1.0, out


def test_a_weaker_bound_is_caught():
    """Planted mistake: the same harness against a copy of the header whose
    bound constants are a third of the real ones must report violations, so
    the adversarial families reach the bound."""
    with tempfile.TemporaryDirectory() as d:
        hdr = open(os.path.join(CSRC, "screen.cuh")).read()
        weak = hdr.replace("constexpr float kC2 = 1.5f * 1.0128f * 264.6f * kEps;",
                           "constexpr float kC2 = 0.5f * 1.0128f * 264.6f * kEps * 0.05f;")
        weak = weak.replace("constexpr float kC1 = 1.5f * 1.0128f * 13.2f * kEps;",
                            "constexpr float kC1 = 0.05f * 1.0128f * 13.2f * kEps;")
        weak = weak.replace("constexpr float kC3 = 1.5f * 1.0128f * 194.0f * kEps;",
                            "constexpr float kC3 = 0.05f * 1.0128f * 194.0f * kEps;")
        assert weak != hdr
        os.makedirs(os.path.join(d, "w"))
        with open(os.path.join(d, "w", "screen.cuh"), "w") as f:
            f.write(weak)
        exe = _build(d, os.path.join(d, "w"))
        rc, out = _run(exe, 100_000, 0)
        assert rc != 0 and "BAD" in out, out


def test_a_weaker_difference_screen_is_caught():
    """Planted mistake: kE64 a millionth of its value lets the difference
    screen claim signs at rounding level, which the FP64 comparison contradicts."""
    with tempfile.TemporaryDirectory() as d:
        hdr = open(os.path.join(CSRC, "screen.cuh")).read()
        weak = hdr.replace("constexpr float kE64 = 4e-15f;", "constexpr float kE64 = 4e-21f;")
        weak = weak.replace("if (!(fabsf(N) - 2.0f * eN > need)) return 0;", "if (!(fabsf(N) > need)) return 0;")
        assert weak != hdr
        os.makedirs(os.path.join(d, "w"))
        with open(os.path.join(d, "w", "screen.cuh"), "w") as f:
            f.write(weak)
        exe = _build(d, os.path.join(d, "w"))
        rc, out = _run(exe, 200_000, 0)
        assert rc != 0 and "BAD diff" in out, out
