// pass_screened.cu -- the fast exact Jacobi pass of Smart Laplacian smoothing.
//
// Same results, bit for bit, as the FP64 pass (Eq. 2 with the accept test of
// Section 3.3.4); what changes is which pipe does the work.  GB300 issues about
// two FP64 operations per SM per clock against ~128 FP32/INT32, so:
//
//  1. The neighbour sums (Eq. 2) are carried out exactly on the integer pipe.
//     Every coordinate of the node's one-ring is a multiple of one power of two
//     u = 2^(F-1075) when the ring's exponents lie in [F, F+4]; the running sum
//     is an int64 multiple of u, rounded to 53 significant bits
//     (round-to-nearest-even) after every addition -- exactly what each FP64
//     addition does.
//  2. The division by the degree uses Markstein's correction (Markstein, IBM J.
//     Res. Dev. 34(1), 1990): q0 = s*y with y = RN(1/N), r = fma(-q0, N, s)
//     (exact), q = fma(r, y, q0), which is the correctly rounded s/N.  Three
//     FP64 operations instead of a full division.
//  3. If the centre equals the node's position bit for bit, q_new == q_old
//     exactly and no quality needs evaluating.
//  4. Otherwise alpha of every incident triangle, before and after the move, is
//     evaluated in FP32 in a frame centred on the node (local coordinates are
//     exact integer differences, rounded once to FP32) together with a
//     rigorous bound on its distance to the exact alpha of the FP64 inputs,
//     wide enough to also cover the FP64 evaluation's own rounding.  When the
//     intervals of q_new and q_old are disjoint the FP64 decision is known.
//  5. Nodes the screen cannot decide (near-ties), or whose ring leaves the
//     fast path's limits, are queued in shared memory and finished by the
//     exact FP64 update, densely packed so the narrow FP64 pipe is not wasted
//     on idle lanes; only the triangles the screen could not rule out as the
//     minimum are evaluated in FP64.
#include <cfloat>

#include "kernels.h"
#include "node_exact.cuh"

namespace sls {

namespace {

constexpr int kFastMax = 16;  // degree and triangle limits of the screened path
__constant__ double c_recip[kFastMax + 1];  // RN(1/N)

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ int bexp(unsigned long long b) { return (int)((b >> 52) & 0x7ffull); }

// +0.0 or a finite normal number (the fast path's domain).
__device__ __forceinline__ bool in_domain(unsigned long long b)
{
    const int e = bexp(b);
    return b == 0ull || (e != 0 && e != 0x7ff);
}

// Value b as an integer multiple of 2^(F-1075); b must be 0 or have its
// exponent in [F, F+4].
__device__ __forceinline__ long long to_frame(unsigned long long b, int F)
{
    if (b == 0ull) return 0ll;
    const long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << (bexp(b) - F);
    return (b >> 63) ? -m : m;
}

// Round an int64 (|S| < 2^63) to 53 significant bits, ties to even: the
// rounding of one FP64 addition whose exact result is S * 2^(F-1075).
__device__ __forceinline__ long long rn53(long long S)
{
    unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    if (a < (1ull << 53)) return S;
    const int sh = 11 - __clzll((long long)a);  // bit length - 53, in 1..10
    const unsigned long long unit = 1ull << sh;
    const unsigned long long rem = a & (unit - 1ull);
    const unsigned long long half = unit >> 1;
    a -= rem;
    if (rem > half || (rem == half && (a & unit))) a += unit;
    return S < 0 ? -(long long)a : (long long)a;
}

// The double S * 2^(F-1075), for S with at most 53 significant bits.
__device__ __forceinline__ double from_frame(long long S, int F)
{
    if (S == 0) return 0.0;
    const unsigned long long sign = S < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
    const int L = 64 - __clzll((long long)a);
    const unsigned long long m = L > 53 ? (a >> (L - 53)) : (a << (53 - L));
    return bitsd(sign | ((unsigned long long)(F + L - 53) << 52) | (m & 0xFFFFFFFFFFFFFull));
}

// Markstein's correctly rounded division by a small integer N (y = RN(1/N)).
__device__ __forceinline__ double div_small(double s, double N, double y)
{
    const double q0 = __dmul_rn(s, y);
    const double r = __fma_rn(-q0, N, s);
    return __fma_rn(r, y, q0);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// Screening constants (unit roundoff e = 2^-24).  For a triangle whose
// vertices' local coordinates are bounded by R, with g = R^2 / s (s the
// computed sum of squared edges), the FP32 alpha differs from the exact alpha
// of the FP64 inputs by at most
//   e * (13.2 |a| + (155.9 + 98 |a|) g) * (1 + 1.1 e (6.1 + 98 g)),
// (edge errors 4.01 e R, cross 45 e R^2, edge sum 6.1 e s + 98 e R^2, FP32
// constant, products and approximate reciprocal 7.1 e |a|), valid for
// g <= kGMax.  The constants carry a further factor 1.5.  Because g >= 1/24
// (every squared edge is at most 8 R^2), half of the resulting bound is at
// least 3e-7: more than the FP64 evaluation's own error (< 2e-15 for
// |alpha| <= 1) plus the FP32 rounding of a +- b and of the comparisons, so
// those need no separate term.
constexpr float kEps = 5.9604645e-8f;
constexpr float kC1 = 1.5f * 1.0065f * 13.2f * kEps;
constexpr float kC2 = 1.5f * 1.0065f * 155.9f * kEps;
constexpr float kC3 = 1.5f * 1.0065f * 98.0f * kEps;
constexpr float kGMax = 1000.0f;
constexpr float kTwoSqrt3f = 3.46410161514f;

// Interval [lo, hi] of the minimum over triangles and the candidate test.
struct MinTrack {
    float minU, minLother, lofBest;
    int best;
    __device__ __forceinline__ void init()
    {
        minU = FLT_MAX;
        minLother = FLT_MAX;
        lofBest = FLT_MAX;
        best = 0;
    }
    __device__ __forceinline__ void add(float a, float b, int t)
    {
        const float U = a + b, L = a - b;
        if (U < minU) {
            minLother = fminf(minLother, lofBest);
            minU = U;
            lofBest = L;
            best = t;
        } else {
            minLother = fminf(minLother, L);
        }
    }
    __device__ __forceinline__ float lo() const { return fminf(minLother, lofBest); }
    __device__ __forceinline__ bool single() const { return minLother > minU; }
};

// FP32 alpha and its bound for the triangle (X, A, B) in that orientation.
__device__ __forceinline__ void screen_alpha(float Xx, float Xy, float Ax, float Ay, float Bx, float By,
                                             float ba2, float R2, float sgn, float &a, float &b)
{
    const float e1x = Ax - Xx, e1y = Ay - Xy, e2x = Bx - Xx, e2y = By - Xy;
    const float cr = fmaf(e1x, e2y, -(e1y * e2x));
    const float s = fmaf(e1x, e1x, fmaf(e1y, e1y, fmaf(e2x, e2x, fmaf(e2y, e2y, ba2))));
    const float inv = __fdividef(1.0f, s);
    a = sgn * kTwoSqrt3f * cr * inv;
    const float g = R2 * inv;
    const float aa = fabsf(a);
    b = fmaf(kC1, aa, fmaf(kC3, aa, kC2) * g);
    if (!(s > 0.0f) || !(g <= kGMax)) {  // degenerate or unscreenable: no information
        a = 0.0f;
        b = FLT_MAX;
    }
}

template <int LAYOUT>
__global__ void __launch_bounds__(512) pass_screened_kernel(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_qn;
    const int nthr = blockDim.x;
    float2 *s_loc = reinterpret_cast<float2 *>(smem_raw);                       // [kFastMax][nthr]
    Deferred *s_q = reinterpret_cast<Deferred *>(s_loc + kFastMax * nthr);      // [2 * nthr]

    if (pass_is_skipped(a.stats, a.q, a.tol_active, a.thr_bits)) return;
    const int tid = threadIdx.x;
    if (blockIdx.x == 0 && tid == 0) a.stats[a.q].executed = 1u;
    if (tid == 0) s_qn = 0;
    __syncthreads();

    unsigned long long best = 0ull, nacc = 0ull, nfb = 0ull;
    float2 *loc = s_loc + tid;
    const int64_t ntiles = (a.n + nthr - 1) / nthr;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t i = tile * nthr + tid;
        bool defer = false;
        Deferred d;
        d.flags = 0u;
        d.cx = 0.0;
        d.cy = 0.0;
        if (i < a.n) {
            d.node = (int32_t)i;
            const uint32_t off = __ldg(a.node_off + i);
            const uint32_t meta = __ldg(a.adj + off);
            if (meta & kMetaFixed) {
                if (a.accept) a.accept[i] = 0;
            } else {
                const uint32_t deg = meta_degree(meta), ntri = meta_ntri(meta);
                const uint32_t *nb = a.adj + off + 1;
                const double2 p = Coords<LAYOUT>::get(a.in, a.n, i);
                const unsigned long long px = dbits(p.x), py = dbits(p.y);
                bool ok = deg <= (uint32_t)kFastMax && ntri <= (uint32_t)kFastMax && in_domain(px) && in_domain(py);
                // exponent window of the ring (zeros impose nothing)
                int hx = px ? bexp(px) : 0, lx = px ? bexp(px) : 2047;
                int hy = py ? bexp(py) : 0, ly = py ? bexp(py) : 2047;
                if (ok) {
                    for (uint32_t k = 0; k < deg; ++k) {
                        const double2 v = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb + k));
                        const unsigned long long vx = dbits(v.x), vy = dbits(v.y);
                        ok = ok && in_domain(vx) && in_domain(vy);
                        if (vx) { hx = max(hx, bexp(vx)); lx = min(lx, bexp(vx)); }
                        if (vy) { hy = max(hy, bexp(vy)); ly = min(ly, bexp(vy)); }
                    }
                }
                const int Fx = hx ? hx - 4 : 1019, Fy = hy ? hy - 4 : 1019;
                ok = ok && lx >= Fx && ly >= Fy && Fx >= 960 && Fx <= 1070 && Fy >= 960 && Fy <= 1070;
                if (!ok) {
                    defer = true;  // exact path computes everything
                } else {
                    // Eq. 2 on the integer pipe, in the stored summation order
                    const long long Mx = to_frame(px, Fx), My = to_frame(py, Fy);
                    const float scx = pow2f(Fx - 1075), scy = pow2f(Fy - 1075);
                    long long Sx = 0, Sy = 0;
                    float R = 0.0f;
                    for (uint32_t k = 0; k < deg; ++k) {
                        const double2 v = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb + k));
                        const long long X = to_frame(dbits(v.x), Fx), Y = to_frame(dbits(v.y), Fy);
                        Sx = k ? rn53(Sx + X) : X;
                        Sy = k ? rn53(Sy + Y) : Y;
                        const float lxf = __ll2float_rn(X - Mx) * scx, lyf = __ll2float_rn(Y - My) * scy;
                        loc[k * nthr] = make_float2(lxf, lyf);
                        R = fmaxf(R, fmaxf(fabsf(lxf), fabsf(lyf)));
                    }
                    const double fd = (double)deg, y = c_recip[deg];
                    const double cx = div_small(from_frame(Sx, Fx), fd, y);
                    const double cy = div_small(from_frame(Sy, Fy), fd, y);
                    d.cx = cx;
                    d.cy = cy;
                    d.flags = kHasCentre;
                    const unsigned long long cbx = dbits(cx), cby = dbits(cy);
                    if (cbx == px && cby == py) {
                        // the centre is the node itself: q_new == q_old exactly
                        const bool acc = !a.strict;
                        Coords<LAYOUT>::put(a.out, a.n, i, p);
                        if (a.accept) a.accept[i] = acc ? 1 : 0;
                        nacc += acc ? 1ull : 0ull;
                    } else if (!((cbx == 0ull || bexp(cbx) >= Fx) && (cby == 0ull || bexp(cby) >= Fy))) {
                        defer = true;
                    } else {
                        const float Cx = __ll2float_rn(to_frame(cbx, Fx) - Mx) * scx;
                        const float Cy = __ll2float_rn(to_frame(cby, Fy) - My) * scy;
                        R = fmaxf(R, fmaxf(fabsf(Cx), fabsf(Cy)));
                        const float R2 = R * R;
                        MinTrack o, nw;
                        o.init();
                        nw.init();
                        for (uint32_t t = 0; t < ntri; ++t) {
                            const uint32_t c = __ldg(nb + deg + t);
                            const float2 A = loc[code_first(c) * nthr];
                            const float2 B = loc[code_second(c) * nthr];
                            const float sgn = code_slot(c) == 1u ? -1.0f : 1.0f;
                            const float bax = B.x - A.x, bay = B.y - A.y;
                            const float ba2 = fmaf(bax, bax, bay * bay);
                            float av, bv;
                            screen_alpha(0.0f, 0.0f, A.x, A.y, B.x, B.y, ba2, R2, sgn, av, bv);
                            o.add(av, bv, (int)t);
                            screen_alpha(Cx, Cy, A.x, A.y, B.x, B.y, ba2, R2, sgn, av, bv);
                            nw.add(av, bv, (int)t);
                        }
                        // q_new and q_old (FP64) lie in [lo, minU] of their side
                        const float new_lo = nw.lo(), new_hi = nw.minU;
                        const float old_lo = o.lo(), old_hi = o.minU;
                        if (R2 >= 1e-30f && R2 <= 1e30f && (new_lo > old_hi || new_hi < old_lo)) {
                            const bool acc = new_lo > old_hi;
                            double2 outp = p;
                            if (acc) {
                                const double dx = __dsub_rn(cx, p.x), dy = __dsub_rn(cy, p.y);
                                const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
                                const unsigned long long b2 = dbits(d2);
                                best = b2 > best ? b2 : best;
                                nacc += 1ull;
                                outp = make_double2(cx, cy);
                            }
                            Coords<LAYOUT>::put(a.out, a.n, i, outp);
                            if (a.accept) a.accept[i] = acc ? 1 : 0;
                        } else {
                            defer = true;
                            d.flags |= (o.single() ? kSingleOld : 0u) | (nw.single() ? kSingleNew : 0u) |
                                       ((uint32_t)o.best << 8) | ((uint32_t)nw.best << 16);
                        }
                    }
                }
            }
        }
        if (defer) {
            const int slot = atomicAdd(&s_qn, 1);
            s_q[slot] = d;
            nfb += 1ull;
        }
        __syncthreads();
        const int qn = s_qn;
        if (qn >= nthr || tile + gridDim.x >= ntiles) {
            for (int k = tid; k < qn; k += nthr) {
                const Deferred e = s_q[k];
                unsigned long long b2;
                bool acc;
                exact_update<LAYOUT>(a, e.node, e.flags, e.cx, e.cy, b2, acc);
                best = b2 > best ? b2 : best;
                nacc += acc ? 1ull : 0ull;
            }
            __syncthreads();
            if (tid == 0) s_qn = 0;
            __syncthreads();
        }
    }
    block_reduce_stats(a.stats + a.q, best, nacc, nfb);
}

bool g_consts_ready = false;

cudaError_t ensure_constants()
{
    if (g_consts_ready) return cudaSuccess;
    double r[kFastMax + 1];
    r[0] = 0.0;
    for (int k = 1; k <= kFastMax; ++k) r[k] = 1.0 / (double)k;
    cudaError_t e = cudaMemcpyToSymbol(c_recip, r, sizeof r);
    if (e != cudaSuccess) return e;
    for (int L = 0; L < 2; ++L) {
        e = cudaFuncSetAttribute(L == 0 ? (const void *)pass_screened_kernel<0> : (const void *)pass_screened_kernel<1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    g_consts_ready = true;
    return cudaSuccess;
}

}  // namespace

size_t screened_smem_bytes(int block)
{
    return (size_t)block * (kFastMax * sizeof(float2) + 2 * sizeof(Deferred));
}

cudaError_t launch_pass_screened(const PassArgs &a, int layout, int block, int grid, cudaStream_t s)
{
    cudaError_t e = ensure_constants();
    if (e != cudaSuccess) return e;
    const size_t smem = screened_smem_bytes(block);
    if (layout == 0) pass_screened_kernel<0><<<grid, block, smem, s>>>(a);
    else pass_screened_kernel<1><<<grid, block, smem, s>>>(a);
    return cudaGetLastError();
}

int pass_screened_occupancy(int layout, int block)
{
    if (ensure_constants() != cudaSuccess) return 1;
    int nb = 0;
    const size_t smem = screened_smem_bytes(block);
    if (layout == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_screened_kernel<0>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_screened_kernel<1>, block, smem);
    return nb > 0 ? nb : 1;
}

}  // namespace sls
