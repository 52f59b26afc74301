// pass_f32.cu -- Smart Laplacian passes in binary32, the paper's precision
// (Section 4).
//
// The coordinates are stored as floats and every step is one binary32
// round-to-nearest operation in the order of the FP64 definition: the
// neighbour sum of Eq. 2 in the stored order, the division by the neighbour
// count, alpha of Section 3.3.1 with the same expression tree, the accept test
// of Section 3.3.4, the squared move.  Nothing here needs screening: the
// exact binary32 evaluation is itself cheap on the FP32 pipe, so one thread
// takes one node from start to end.
#include <cfloat>

#include "kernels.h"

namespace sls {

namespace {

template <int LAYOUT>
struct Coords32;

template <>
struct Coords32<0> {  // AoS: one float2 per node
    static __device__ __forceinline__ float2 get(const float *p, int64_t, int64_t i)
    {
        return __ldg(reinterpret_cast<const float2 *>(p) + i);
    }
    static __device__ __forceinline__ void put(float *p, int64_t, int64_t i, float2 v)
    {
        reinterpret_cast<float2 *>(p)[i] = v;
    }
};

template <>
struct Coords32<1> {  // SoA: x[n] then y[n]
    static __device__ __forceinline__ float2 get(const float *p, int64_t n, int64_t i)
    {
        return make_float2(__ldg(p + i), __ldg(p + n + i));
    }
    static __device__ __forceinline__ void put(float *p, int64_t n, int64_t i, float2 v)
    {
        p[i] = v.x;
        p[n + i] = v.y;
    }
};

// alpha of the triangle (a, b, c) in stored order, in binary32, with the
// tree of the FP64 definition; every operation an explicit round-to-nearest
// intrinsic (no contraction).  K is the float nearest to 2 sqrt(3).
__device__ __forceinline__ float alpha_f32(float ax, float ay, float bx, float by, float cx, float cy)
{
    const float kTwoSqrt3 = 3.46410161514f;
    const float e1x = __fsub_rn(bx, ax), e1y = __fsub_rn(by, ay);
    const float e2x = __fsub_rn(cx, ax), e2y = __fsub_rn(cy, ay);
    const float e3x = __fsub_rn(cx, bx), e3y = __fsub_rn(cy, by);
    const float cross = __fsub_rn(__fmul_rn(e1x, e2y), __fmul_rn(e1y, e2x));
    const float l1 = __fadd_rn(__fmul_rn(e1x, e1x), __fmul_rn(e1y, e1y));
    const float l2 = __fadd_rn(__fmul_rn(e2x, e2x), __fmul_rn(e2y, e2y));
    const float l3 = __fadd_rn(__fmul_rn(e3x, e3x), __fmul_rn(e3y, e3y));
    const float s = __fadd_rn(__fadd_rn(l1, l2), l3);
    return s > 0.0f ? __fdiv_rn(__fmul_rn(kTwoSqrt3, cross), s) : 0.0f;
}

// alpha of an incident triangle (node i, neighbours A and B) with node i at
// x, in the triangle's stored vertex order (i in slot `slot`, A before B).
// The tree of alpha_f32 rewritten with u = x - A, w = x - B, v = B - A: every
// edge of the stored order is one of +-u, +-w, +-v, and negation commutes
// with rounding, so
//   slot 0: cross = u x w,     s = (|u|^2 + |w|^2) + |v|^2
//   slot 1: cross = u x v,     s = (|u|^2 + |v|^2) + |w|^2
//   slot 2: cross = -(u x v),  s = (|v|^2 + |u|^2) + |w|^2 (the same sum)
// give bit for bit the values of alpha_f32 on the reordered points.  v and
// |v|^2 are shared by both positions of node i; no lane branches on slot.
__device__ __forceinline__ float alpha_uvw(uint32_t slot, float2 x, float2 A, float2 B, float2 v, float lv)
{
    const float kTwoSqrt3 = 3.46410161514f;
    const float2 u = make_float2(__fsub_rn(x.x, A.x), __fsub_rn(x.y, A.y));
    const float2 w = make_float2(__fsub_rn(x.x, B.x), __fsub_rn(x.y, B.y));
    const float lu = __fadd_rn(__fmul_rn(u.x, u.x), __fmul_rn(u.y, u.y));
    const float lw = __fadd_rn(__fmul_rn(w.x, w.x), __fmul_rn(w.y, w.y));
    const bool s0 = slot == 0u;
    const float2 z = s0 ? w : v;
    float cross = __fsub_rn(__fmul_rn(u.x, z.y), __fmul_rn(u.y, z.x));
    cross = slot == 2u ? -cross : cross;
    const float s = __fadd_rn(__fadd_rn(lu, s0 ? lw : lv), s0 ? lv : lw);
    return s > 0.0f ? __fdiv_rn(__fmul_rn(kTwoSqrt3, cross), s) : 0.0f;
}

template <int LAYOUT>
__device__ __forceinline__ float alpha_at(const float *in, int64_t n, const uint32_t *nb, uint32_t code, float2 x)
{
    const float2 A = Coords32<LAYOUT>::get(in, n, __ldg(nb + code_first(code)));
    const float2 B = Coords32<LAYOUT>::get(in, n, __ldg(nb + code_second(code)));
    switch (code_slot(code)) {
    case 0: return alpha_f32(x.x, x.y, A.x, A.y, B.x, B.y);
    case 1: return alpha_f32(A.x, A.y, x.x, x.y, B.x, B.y);
    default: return alpha_f32(A.x, A.y, B.x, B.y, x.x, x.y);
    }
}

// Rings up to this size live in shared memory (larger ones are read from
// global memory).  12 slots keep five blocks' buffers within the 132 KB
// shared-memory carve-out, which leaves the gathers about twice the L1 of
// 16 slots (2.4% faster on jittered grids; a Delaunay mesh of random points
// has about 1.4 nodes in 10,000 above 12).
constexpr int kRingMax = 12;

// One pass over every node (a.order null) or over the listed nodes (one
// colour class of Form B, in place).  a.in / a.out hold floats.  Each thread
// keeps its node's ring in its own column of a shared buffer (stride: block);
// nodes with larger rings read their neighbours from global memory.
template <int LAYOUT>
__global__ void __launch_bounds__(256) pass_f32_kernel(PassArgs a)
{
    __shared__ float2 s_ring[kRingMax * 256];
    if (pass_is_skipped(a.stats, a.q, a.tol_active, a.thr_bits)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.stats[a.q].executed = 1u;
    const float *in = reinterpret_cast<const float *>(a.in);
    float *out = reinterpret_cast<float *>(a.out);
    float2 *ring = s_ring + threadIdx.x;
    const int rs = blockDim.x;

    unsigned best = 0u;  // bits of the largest squared move (non-negative floats order as integers)
    unsigned long long nacc = 0ull;
    const int64_t cnt = a.order ? a.norder : (a.ranged ? a.count : a.n);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += stride) {
        const int64_t i = a.order ? (int64_t)__ldg(a.order + j) : a.first + j;
        const uint32_t off = __ldg(a.node_off + i);
        const uint32_t meta = __ldg(a.adj + off);
        if (meta & kMetaFixed) {
            if (a.accept) a.accept[i] = 0;
            continue;
        }
        const uint32_t deg = meta_degree(meta), ntri = meta_ntri(meta);
        const uint32_t *nb = a.adj + off + 1;
        const float2 p = Coords32<LAYOUT>::get(in, a.n, i);
        float2 c;
        float q_old = FLT_MAX, q_new = FLT_MAX;
        bool tie;
        if (deg <= (uint32_t)kRingMax) {
            // Eq. 2 in the stored order; the ring goes to shared memory
            float2 v = Coords32<LAYOUT>::get(in, a.n, __ldg(nb));
            ring[0] = v;
            float sx = v.x, sy = v.y;
            for (uint32_t k = 1; k < deg; ++k) {
                v = Coords32<LAYOUT>::get(in, a.n, __ldg(nb + k));
                ring[k * rs] = v;
                sx = __fadd_rn(sx, v.x);
                sy = __fadd_rn(sy, v.y);
            }
            const float fd = (float)deg;
            c = make_float2(__fdiv_rn(sx, fd), __fdiv_rn(sy, fd));
            tie = __float_as_uint(c.x) == __float_as_uint(p.x) && __float_as_uint(c.y) == __float_as_uint(p.y);
            if (!tie) {
                for (uint32_t t = 0; t < ntri; ++t) {
                    const uint32_t code = __ldg(nb + deg + t);
                    const float2 A = ring[code_first(code) * rs];
                    const float2 B = ring[code_second(code) * rs];
                    const float2 vv = make_float2(__fsub_rn(B.x, A.x), __fsub_rn(B.y, A.y));
                    const float lv = __fadd_rn(__fmul_rn(vv.x, vv.x), __fmul_rn(vv.y, vv.y));
                    const float qo = alpha_uvw(code_slot(code), p, A, B, vv, lv);
                    const float qn = alpha_uvw(code_slot(code), c, A, B, vv, lv);
                    q_old = (t == 0u || qo < q_old) ? qo : q_old;  // first wins, as in the definition
                    q_new = (t == 0u || qn < q_new) ? qn : q_new;
                }
            }
        } else {
            float2 v = Coords32<LAYOUT>::get(in, a.n, __ldg(nb));
            float sx = v.x, sy = v.y;
            for (uint32_t k = 1; k < deg; ++k) {
                v = Coords32<LAYOUT>::get(in, a.n, __ldg(nb + k));
                sx = __fadd_rn(sx, v.x);
                sy = __fadd_rn(sy, v.y);
            }
            const float fd = (float)deg;
            c = make_float2(__fdiv_rn(sx, fd), __fdiv_rn(sy, fd));
            tie = __float_as_uint(c.x) == __float_as_uint(p.x) && __float_as_uint(c.y) == __float_as_uint(p.y);
            if (!tie) {
                for (uint32_t t = 0; t < ntri; ++t) {
                    const uint32_t code = __ldg(nb + deg + t);
                    const float qo = alpha_at<LAYOUT>(in, a.n, nb, code, p);
                    const float qn = alpha_at<LAYOUT>(in, a.n, nb, code, c);
                    q_old = (t == 0u || qo < q_old) ? qo : q_old;
                    q_new = (t == 0u || qn < q_new) ? qn : q_new;
                }
            }
        }
        // a tie (the centre is the node itself) means q_new == q_old
        const bool ok = tie ? !a.strict : (a.strict ? (q_new > q_old) : (q_new >= q_old));
        float2 o = p;
        if (ok) {
            const float dx = __fsub_rn(c.x, p.x), dy = __fsub_rn(c.y, p.y);
            const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
            best = max(best, __float_as_uint(d2));
            nacc += 1ull;
            o = c;
        }
        Coords32<LAYOUT>::put(out, a.n, i, o);
        if (a.accept) a.accept[i] = ok ? 1 : 0;
    }
    // widened exactly to double, so the pass records compare like FP64 ones
    const unsigned long long b64 = (unsigned long long)__double_as_longlong((double)__uint_as_float(best));
    block_reduce_stats(a.stats + a.q, b64, nacc, 0ull);
}

__global__ void copy_back_f32_kernel(const float *__restrict__ src, float *__restrict__ dst, int64_t count,
                                     const PassStats *stats, int q)
{
    if (stats[q].executed == 0u) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride)
        dst[k] = __ldg(src + k);
}

// interleaved doubles -> floats in the mesh's layout (round to nearest)
__global__ void narrow_kernel(const double2 *__restrict__ aos, float *dst, int64_t n, int layout)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 v = __ldg(aos + i);
        const float x = __double2float_rn(v.x), y = __double2float_rn(v.y);
        if (layout == 0) {
            reinterpret_cast<float2 *>(dst)[i] = make_float2(x, y);
        } else {
            dst[i] = x;
            dst[n + i] = y;
        }
    }
}

// floats in the mesh's layout -> interleaved doubles (exact)
__global__ void widen_kernel(const float *__restrict__ src, double2 *aos, int64_t n, int layout)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float x, y;
        if (layout == 0) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(src) + i);
            x = v.x;
            y = v.y;
        } else {
            x = __ldg(src + i);
            y = __ldg(src + n + i);
        }
        aos[i] = make_double2((double)x, (double)y);
    }
}

}  // namespace

cudaError_t launch_pass_f32(const PassArgs &a, int layout, int block, int grid, cudaStream_t s)
{
    if (layout == 0) pass_f32_kernel<0><<<grid, block, 0, s>>>(a);
    else pass_f32_kernel<1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int pass_f32_occupancy(int layout, int block)
{
    int nb = 0;
    if (layout == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_f32_kernel<0>, block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_f32_kernel<1>, block, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_copy_back_f32(const float *src, float *dst, int64_t count, const PassStats *stats, int q,
                                 int grid, cudaStream_t s)
{
    copy_back_f32_kernel<<<grid, 256, 0, s>>>(src, dst, count, stats, q);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const double *aos, float *dst, int64_t n, int layout, int grid, cudaStream_t s)
{
    narrow_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const double2 *>(aos), dst, n, layout);
    return cudaGetLastError();
}

cudaError_t launch_widen(const float *src, double *aos, int64_t n, int layout, int grid, cudaStream_t s)
{
    widen_kernel<<<grid, 256, 0, s>>>(src, reinterpret_cast<double2 *>(aos), n, layout);
    return cudaGetLastError();
}

}  // namespace sls
