// device.cuh -- device-side types and helpers shared by the slsmooth kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sls {

// Per-pass statistics, one record per pass of an sls_smooth call (or per pass
// and mesh in the batched form).  Written with atomics by the pass kernel.
struct PassStats {
    unsigned long long maxd2_bits;  // bits of the largest squared move (>= 0, so bit order = value order)
    unsigned long long nacc;        // accepted free nodes
    unsigned long long fallbacks;   // accept tests redone in FP64 by the screened kernel
    unsigned int executed;          // 1 once the pass ran (0: skipped after convergence)
    unsigned int nodes_skipped;     // node updates not recomputed (unchanged inputs)
};

// Arguments of one Jacobi pass over one mesh.
struct PassArgs {
    const double *in;          // coordinates X^q   (AoS: x0 y0 x1 y1 ...; SoA: x[n] then y[n])
    double *out;               // coordinates X^q+1 (free nodes written; fixed nodes are never written)
    const uint32_t *node_off;  // n+1 word offsets into adj
    const uint32_t *adj;       // per-node words: meta, neighbours, triangle codes
    int64_t n;
    const uint32_t *order;     // nullptr: every node in index order; else the nodes to update
    int64_t norder;            // (one colour class of Form B) and their number
    int ranged;                // 1 (order null): only the nodes first .. first + count - 1
    int64_t first, count;      // (a contiguous colour class of a renumbered Form-B mesh)
    PassStats *stats;          // stats[q] receives this pass
    int q;                     // pass index within the call
    int strict;                // 1: accept iff q_new > q_old
    int tol_active;            // 1: skip the pass when pass q-1 met the tolerance or was skipped
    unsigned long long thr_bits;  // bits of (tol * D)^2
    uint8_t *accept;           // n decisions, or nullptr
    // Skipping of unchanged tiles (tiles of 32 consecutive nodes; all null
    // and skip = 0 when the mesh does not use it).  A tile whose nodes and
    // whose nodes' neighbours all kept their coordinates in the previous pass
    // has the same inputs as then, so its update is the identity: its nodes
    // keep their coordinates (already in `out`, two passes old and equal) and
    // their decisions.
    const uint2 *halo;         // kHaloEntries (tile, node mask) pairs per tile: itself and every
                               // tile holding a neighbour of one of its nodes; (kHaloNever, 0)
                               // first marks a tile that is never skipped
    const uint32_t *chg_prev;  // per tile: nodes whose coordinates changed in the previous pass
    uint32_t *chg_cur;         // the same, written by this pass
    uint32_t *accm;            // per tile: nodes accepted the last time the tile was computed
    int skip;                  // 1: unchanged tiles may be skipped in this pass
};

constexpr int kHaloEntries = 16;
constexpr uint32_t kHaloNever = 0xffffffffu;

// One mesh (job) of the batched and served forms.
struct JobDesc {
    double *xy[2];             // the job's two coordinate arrays
    const uint32_t *node_off;  // n+1
    const uint32_t *adj;
    int64_t n;
    PassStats *stats;          // one record per pass of the job
    unsigned long long thr_bits;
    int32_t strict, tol_active;
    int32_t max_iter;          // passes to run at most
    int32_t base_round;        // the job's pass q runs in round base_round + q
    int32_t cur0;              // which array holds the job's starting coordinates
    int32_t pad;
    uint8_t *accept;           // n decisions, or nullptr
};

// 32 consecutive nodes [first, first + 32) of one job.
struct WarpTask {
    int32_t job;
    int32_t first;
};

constexpr uint32_t kMetaFixed = 0x80000000u;

__device__ __forceinline__ uint32_t meta_degree(uint32_t meta) { return meta & 0xffffu; }
__device__ __forceinline__ uint32_t meta_ntri(uint32_t meta) { return (meta >> 16) & 0x7fffu; }
__device__ __forceinline__ uint32_t code_slot(uint32_t c) { return c >> 30; }
__device__ __forceinline__ uint32_t code_first(uint32_t c) { return (c >> 15) & 0x7fffu; }
__device__ __forceinline__ uint32_t code_second(uint32_t c) { return c & 0x7fffu; }

// A pass is skipped when the tolerance is on and the previous pass either
// was skipped or already moved no node by (tol * D) or more.
__device__ __forceinline__ bool pass_is_skipped(const PassStats *stats, int q, int tol_active,
                                                unsigned long long thr_bits)
{
    if (!tol_active || q == 0) return false;
    const PassStats &p = stats[q - 1];
    return p.executed == 0u || p.maxd2_bits < thr_bits;
}

// Coordinate access for the two layouts.
template <int LAYOUT>
struct Coords;

template <>
struct Coords<0> {  // AoS: one double2 per node
    static __device__ __forceinline__ double2 get(const double *p, int64_t, int64_t i)
    {
        return __ldg(reinterpret_cast<const double2 *>(p) + i);
    }
    static __device__ __forceinline__ void put(double *p, int64_t, int64_t i, double2 v)
    {
        reinterpret_cast<double2 *>(p)[i] = v;
    }
};

template <>
struct Coords<1> {  // SoA: x[n] then y[n]
    static __device__ __forceinline__ double2 get(const double *p, int64_t n, int64_t i)
    {
        return make_double2(__ldg(p + i), __ldg(p + n + i));
    }
    static __device__ __forceinline__ void put(double *p, int64_t n, int64_t i, double2 v)
    {
        p[i] = v.x;
        p[n + i] = v.y;
    }
};

// The same coordinates as raw 64-bit patterns.  Code that only moves or
// inspects coordinates uses these, so no value is ever held in an FP64
// register (the compiler copies FP64 registers with FP64-pipe instructions).
template <int LAYOUT>
struct CoordBits;

template <>
struct CoordBits<0> {
    static __device__ __forceinline__ ulonglong2 get(const double *p, int64_t, int64_t i)
    {
        return __ldg(reinterpret_cast<const ulonglong2 *>(p) + i);
    }
    static __device__ __forceinline__ void put(double *p, int64_t, int64_t i, ulonglong2 v)
    {
        reinterpret_cast<ulonglong2 *>(p)[i] = v;
    }
};

template <>
struct CoordBits<1> {
    static __device__ __forceinline__ ulonglong2 get(const double *p, int64_t n, int64_t i)
    {
        const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
        return make_ulonglong2(__ldg(q + i), __ldg(q + n + i));
    }
    static __device__ __forceinline__ void put(double *p, int64_t n, int64_t i, ulonglong2 v)
    {
        unsigned long long *q = reinterpret_cast<unsigned long long *>(p);
        q[i] = v.x;
        q[n + i] = v.y;
    }
};

// Lee and Lo's alpha of the triangle (a, b, c) in its stored vertex order:
// 2*sqrt(3) * cross / ((|e1|^2 + |e2|^2) + |e3|^2), e1 = b-a, e2 = c-a,
// e3 = c-b, cross = e1x*e2y - e1y*e2x; 0 when the edge sum is not positive.
// Every operation is an explicit round-to-nearest intrinsic, so nothing is
// contracted into an FMA.
__device__ __forceinline__ double alpha_fp64(double ax, double ay, double bx, double by, double cx,
                                             double cy)
{
    const double kTwoSqrt3 = 3.4641016151377544;  // nearest double to 2*sqrt(3)
    double e1x = __dsub_rn(bx, ax), e1y = __dsub_rn(by, ay);
    double e2x = __dsub_rn(cx, ax), e2y = __dsub_rn(cy, ay);
    double e3x = __dsub_rn(cx, bx), e3y = __dsub_rn(cy, by);
    double cross = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
    double l1 = __dadd_rn(__dmul_rn(e1x, e1x), __dmul_rn(e1y, e1y));
    double l2 = __dadd_rn(__dmul_rn(e2x, e2x), __dmul_rn(e2y, e2y));
    double l3 = __dadd_rn(__dmul_rn(e3x, e3x), __dmul_rn(e3y, e3y));
    double s = __dadd_rn(__dadd_rn(l1, l2), l3);
    return s > 0.0 ? __ddiv_rn(__dmul_rn(kTwoSqrt3, cross), s) : 0.0;
}

// Block-wide reduction of (max of d2 bits, accepted count, fallbacks) into
// stats with one atomic each per block.  All threads of the block must call it.
__device__ __forceinline__ void block_reduce_stats(PassStats *st, unsigned long long d2_bits,
                                                   unsigned long long nacc,
                                                   unsigned long long nfb)
{
    __shared__ unsigned long long s_max[32], s_acc[32], s_fb[32];
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long m2 = __shfl_xor_sync(0xffffffffu, d2_bits, o);
        d2_bits = m2 > d2_bits ? m2 : d2_bits;
        nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
    }
    if (lane == 0) {
        s_max[warp] = d2_bits;
        s_acc[warp] = nacc;
        s_fb[warp] = nfb;
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned nw = (blockDim.x + 31u) >> 5;
        d2_bits = lane < nw ? s_max[lane] : 0ull;
        nacc = lane < nw ? s_acc[lane] : 0ull;
        nfb = lane < nw ? s_fb[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long m2 = __shfl_xor_sync(0xffffffffu, d2_bits, o);
            d2_bits = m2 > d2_bits ? m2 : d2_bits;
            nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
            nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
        }
        if (lane == 0) {
            if (d2_bits) atomicMax(&st->maxd2_bits, d2_bits);
            if (nacc) atomicAdd(&st->nacc, nacc);
            if (nfb) atomicAdd(&st->fallbacks, nfb);
        }
    }
}

}  // namespace sls
