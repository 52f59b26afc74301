// screen.cuh -- the FP32 screen of the accept test (Section 3.3.4) used by
// the screened pass: float head/tail splits of the FP64 coordinates, the
// local frame centred on the node, alpha in FP32 with a rigorous bound on its
// distance to the FP64 alpha, and a second screen on the sign of
// alpha(centre) - alpha(node) taken straight from the move.
//
// Compiles for the host too, so the CPU tests run this code against alpha
// evaluated in binary128 and in the FP64 expression tree on adversarial
// triangles.  On the host the approximate reciprocal of the device
// (__fdividef(1, s), at most 2 ulp off for 2^-126 < s < 2^126) is stood in
// for by SLS_SCREEN_HOST_RCP, which a test may define to move the result by
// up to 2 ulp either way.
#pragma once

#include <float.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define SLS_SC_HD __host__ __device__ __forceinline__
#else
#define SLS_SC_HD static inline
#endif

#ifndef SLS_SCREEN_HOST_RCP
#define SLS_SCREEN_HOST_RCP(s) (1.0f / (s))
#endif

namespace sls {
namespace scr {

SLS_SC_HD float u2f(uint32_t u)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, sizeof f);
    return f;
#endif
}

SLS_SC_HD uint32_t f2u(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
#endif
}

// 1/s to within 2 ulp (device: the approximate division).
SLS_SC_HD float rcp_approx(float s)
{
#ifdef __CUDA_ARCH__
    return __fdividef(1.0f, s);
#else
    return SLS_SCREEN_HOST_RCP(s);
#endif
}

// Splits the double with bit pattern b into a float head (its sign, exponent
// and top 24 significant bits) and a float tail (the next 23 bits), with
// integer operations only; head + tail is within 2^-46 |x| of x.  Returns
// false outside [2^-80, 2^127) in magnitude (zero is allowed) or for
// subnormal, infinite or NaN values.
SLS_SC_HD bool head_tail(unsigned long long b, float &hd, float &tl)
{
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned e = (hw >> 20) & 0x7ffu;
    const bool zero = (hw & 0x7fffffffu) == 0u && lw == 0u;
    const unsigned sign = hw & 0x80000000u;
    const float h = u2f(sign | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // tail bits 28..6 of the low word, value t * 2^(E - 46): exact in FP32
    const float t = u2f(0x4b000000u | ((lw >> 6) & 0x7fffffu)) - 8388608.0f;
    const float l = u2f(f2u(t * u2f((e - 942u) << 23)) | sign);
    hd = zero ? 0.0f : h;
    tl = zero ? 0.0f : l;
    return zero || (e - 943u <= 206u);  // [2^-80, 2^127) in magnitude, normal
}

// FP32 value of a double, truncated to 24 significant bits (relative error
// below 2^-23), built with integer operations; zero outside the float range.
SLS_SC_HD float trunc_float(unsigned long long b)
{
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned e = (hw >> 20) & 0x7ffu;
    const float f = u2f((hw & 0x80000000u) | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    return e - 897u <= 253u ? f : 0.0f;
}

// Screening constants (unit roundoff e = 2^-24).  A local coordinate of a
// neighbour carries an error below 2e|X| + 2^-44 M (head/tail truncation; M
// bounds the node's coordinate magnitude plus the ring's extent), which is
// below 3e R wherever R >= 2^-20 M; the screen requires that.  The centre's
// local coordinate is within 2e of its exact value (relative).  For a
// triangle whose three vertices' local coordinates are bounded by R, with
// g = R^2 / s (s the computed sum of squared edges), the FP32 alpha differs
// from the exact alpha of the FP64 inputs by at most
//   e * (13.2 |a| + (264.6 + 194 |a|) g) * (1 + 1.1 e (6.1 + 194 g)),
// (edge errors 8 e R; cross 76.4 e R^2; edge sum 6.1 e s + 194 e R^2; FP32
// constant, products and approximate reciprocal 7.1 e |a|), valid for
// g <= kGMax, where the last factor is at most 1.0128.  The constants carry a
// further factor 1.5.  Because g >= 1/24 (every squared edge is at most
// 8 R^2), half of the resulting bound exceeds 8e-7: more than the FP64
// evaluation's own error (< 2e-15 for |alpha| <= 1) plus the FP32 rounding of
// a +- b and of the comparisons, so those need no separate term.
constexpr float kEps = 5.9604645e-8f;
constexpr float kC1 = 1.5f * 1.0128f * 13.2f * kEps;
constexpr float kC2 = 1.5f * 1.0128f * 264.6f * kEps;
constexpr float kC3 = 1.5f * 1.0128f * 194.0f * kEps;
constexpr float kGMax = 1000.0f;
constexpr float kTwoSqrt3f = 3.46410161514f;
constexpr float kLocalRange = 1048576.0f;  // 2^20: R * 2^20 >= M keeps the head/tail error below e R

// Offset of a neighbour (bit patterns bx, by) from the node whose head/tail
// splits are (phx, plx), (phy, ply); ok &= both splits are valid.
SLS_SC_HD void local_offset(unsigned long long bx, unsigned long long by, float phx, float plx, float phy,
                            float ply, float &Lx, float &Ly, bool &ok)
{
    float hx, lx, hy, ly;
    ok = head_tail(bx, hx, lx) & head_tail(by, hy, ly);
    Lx = (hx - phx) + (lx - plx);
    Ly = (hy - phy) + (ly - ply);
}

// Whether the local frame of a node is usable: rmin / rmax the smallest and
// largest local coordinate magnitude of its neighbours (largest including the
// centre's offset), M bounding the node's coordinate magnitude plus rmax.
SLS_SC_HD bool frame_ok(float rmin, float rmax, float M)
{
    return (rmin >= 1e-14f) & (rmax <= 1e15f) & (rmin * kLocalRange >= M);
}

// FP32 alpha of the triangle (X, A, B) for the screen (sk: orientation sign
// times 2 sqrt(3); ba2 = |B - A|^2); sv receives the edge sum.  The second
// candidate loop of the kernel calls it again and gets the same bits.
SLS_SC_HD float screen_alpha(float Xx, float Xy, float Ax, float Ay, float Bx, float By, float ba2, float sk,
                             float &sv)
{
    const float e1x = Ax - Xx, e1y = Ay - Xy, e2x = Bx - Xx, e2y = By - Xy;
    const float cr = fmaf(e1x, e2y, -(e1y * e2x));
    sv = fmaf(e1x, e1x, fmaf(e1y, e1y, fmaf(e2x, e2x, fmaf(e2y, e2y, ba2))));
    return sk * cr * rcp_approx(sv);
}

// |B - A|^2 in FP32, shared by both sides of one triangle.
SLS_SC_HD float edge_ba2(float Ax, float Ay, float Bx, float By)
{
    const float bax = Bx - Ax, bay = By - Ay;
    return fmaf(bax, bax, bay * bay);
}

// Whether one side's bound applies: smallest edge sum positive, g = R^2 / s
// at most kGMax, largest |alpha| at most 2.
SLS_SC_HD bool bound_ok(float smin, float g, float amax)
{
    return (smin > 0.0f) & (g <= kGMax) & (amax <= 2.0f);
}

// g = R^2 / s of one side (R its largest local coordinate, s its smallest
// edge sum).
SLS_SC_HD float side_g(float R, float smin) { return R * R * rcp_approx(smin); }

// The bound of one side: every FP64 alpha of the side's triangles lies within
// it of the triangle's FP32 alpha.
SLS_SC_HD float side_bound(float amax, float g) { return fmaf(kC1, amax, fmaf(kC3, amax, kC2) * g); }

// Second screen, for a node whose two minima are attained by the same single
// triangle (X, A, B) (X = 0 before the move, X = C after it; sgn gives the
// stored orientation).  Then q_new - q_old (FP64) differs from the exact
// alpha(C) - alpha(0) by at most 2 * kE64, and that exact difference is
//   sgn * K * N / (s_new * s_old),  N = dcr * s_old - cr_old * ds,
// with dcr = C x (A - B) and ds = 2|C|^2 - 2 C.(A + B) computed directly from
// the move (no cancellation between two nearly equal qualities).  Error
// budget (e = 2^-24; A, B within 3 e R, C within 2 e |C|; R >= every local
// coordinate of the triangle and the centre, r >= |C| components): dcr
// 32 e r R, ds 100 e r R, cr_old 16 e R^2, s_old 170 e R^2, s_new 280 e R^2,
// and the roundings of N.  kE64 bounds |FP64 alpha - exact alpha| (about 14.2
// units of 2^-53 for |alpha| <= 1, second-order terms included with margin).
// Returns +1 when q_new > q_old certainly, -1 when q_new < q_old certainly,
// 0 otherwise.
constexpr float kE64 = 4e-15f;

SLS_SC_HD int diff_screen(float Ax, float Ay, float Bx, float By, float Cx, float Cy, float sgn, float M2)
{
    const float R = fmaxf(fmaxf(fmaxf(fabsf(Ax), fabsf(Ay)), fmaxf(fabsf(Bx), fabsf(By))),
                          fmaxf(fabsf(Cx), fabsf(Cy)));
    const float r = fmaxf(fabsf(Cx), fabsf(Cy));
    if (!(R >= 1e-6f && R <= 1e7f)) return 0;  // keep every product a normal float
    if (!(R * R * (kLocalRange * kLocalRange) >= M2)) return 0;
    const float bax = Bx - Ax, bay = By - Ay;
    const float ba2 = fmaf(bax, bax, bay * bay);
    const float cro = fmaf(Ax, By, -(Ay * Bx));
    const float so = fmaf(Ax, Ax, fmaf(Ay, Ay, fmaf(Bx, Bx, fmaf(By, By, ba2))));
    const float ax = Ax - Cx, ay = Ay - Cy, bx = Bx - Cx, by = By - Cy;
    const float sn = fmaf(ax, ax, fmaf(ay, ay, fmaf(bx, bx, fmaf(by, by, ba2))));
    const float dabx = Ax - Bx, daby = Ay - By;
    const float dcr = fmaf(Cx, daby, -(Cy * dabx));
    const float sabx = Ax + Bx, saby = Ay + By;
    const float t = fmaf(Cx, sabx, Cy * saby);
    const float c2 = fmaf(Cx, Cx, Cy * Cy);
    const float ds = 2.0f * (c2 - t);
    const float N = fmaf(dcr, so, -(cro * ds));
    const float rR = r * R, R2 = R * R;
    const float e_dcr = 32.0f * kEps * rR, e_ds = 100.0f * kEps * rR;
    const float e_cro = 16.0f * kEps * R2, e_so = 170.0f * kEps * R2, e_sn = 280.0f * kEps * R2;
    if (!(so > e_so && sn > e_sn)) return 0;  // degenerate: no information
    const float adcr = fabsf(dcr), ads = fabsf(ds), acro = fabsf(cro);
    const float eN = e_dcr * so + (adcr + e_dcr) * e_so + e_cro * ads + (acro + e_cro) * e_ds +
                     kEps * (adcr * so + 2.0f * acro * ads);
    const float need = (2.02f * kE64 / kTwoSqrt3f) * (sn + e_sn) * (so + e_so);
    if (!(fabsf(N) - 2.0f * eN > need)) return 0;
    return ((N > 0.0f) == (sgn > 0.0f)) ? 1 : -1;
}

}  // namespace scr
}  // namespace sls
