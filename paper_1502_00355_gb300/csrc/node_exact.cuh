// node_exact.cuh -- the FP64 node update (Eq. 2 with the accept test of
// Section 3.3.4), used whole by the plain FP64 kernel and, restricted to the
// candidate triangles, by the screened kernel for nodes its FP32 screen could
// not decide.
#pragma once

#include "device.cuh"

namespace sls {

// Flags of a deferred node (screened kernel -> exact path).
constexpr uint32_t kHasCentre = 1u;   // cx, cy hold the node's centre
constexpr uint32_t kMasked = 2u;      // masks name every triangle that can attain q_old / q_new

struct Deferred {
    int32_t node;
    uint32_t flags;
    uint32_t masks;  // bits 0..15: candidates for q_old, bits 16..31: for q_new
    uint32_t pad;
    unsigned long long cx, cy;  // the centre, as FP64 bit patterns
};

// alpha of incident triangle `code` of node i with node i placed at (x, y).
template <int LAYOUT>
__device__ __forceinline__ double alpha_with(const PassArgs &a, const uint32_t *nb, uint32_t code,
                                             double x, double y)
{
    const double2 A = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb + code_first(code)));
    const double2 B = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb + code_second(code)));
    switch (code_slot(code)) {
    case 0: return alpha_fp64(x, y, A.x, A.y, B.x, B.y);
    case 1: return alpha_fp64(A.x, A.y, x, y, B.x, B.y);
    default: return alpha_fp64(A.x, A.y, B.x, B.y, x, y);
    }
}

// Exact update of free node i.  Without kHasCentre the centre is computed
// here (neighbour sum in stored order, then IEEE division).  q_old / q_new are
// the minima over all incident triangles or, with kMasked, over the triangles
// in the masks: the screen proved every other triangle's FP64 alpha larger
// than some masked one, so the minimum is the same.  Writes the node and its
// decision; returns the squared move bits (0 if not accepted), whether it was
// accepted and whether its coordinates changed.
template <int LAYOUT>
__device__ __forceinline__ void exact_update(const PassArgs &a, int64_t i, uint32_t flags, uint32_t masks,
                                             unsigned long long cxb, unsigned long long cyb,
                                             unsigned long long &d2_bits, bool &accepted, bool &moved)
{
    double cx = __longlong_as_double((long long)cxb), cy = __longlong_as_double((long long)cyb);
    const uint32_t off = __ldg(a.node_off + i);
    const uint32_t meta = __ldg(a.adj + off);
    const uint32_t deg = meta_degree(meta), ntri = meta_ntri(meta);
    const uint32_t *nb = a.adj + off + 1;
    const double2 p = Coords<LAYOUT>::get(a.in, a.n, i);

    if (!(flags & kHasCentre)) {
        double2 v = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb));
        double sx = v.x, sy = v.y;
        for (uint32_t k = 1; k < deg; ++k) {
            v = Coords<LAYOUT>::get(a.in, a.n, __ldg(nb + k));
            sx = __dadd_rn(sx, v.x);
            sy = __dadd_rn(sy, v.y);
        }
        const double fd = (double)deg;
        cx = __ddiv_rn(sx, fd);
        cy = __ddiv_rn(sy, fd);
    }

    double q_old = 0.0, q_new = 0.0;
    if ((flags & kMasked) && ntri <= 16u) {
        // Each lane walks its own candidates, so a warp runs as many
        // evaluations as its busiest lane has candidates, not one per triangle.
        // Bits at or above ntri never name a triangle of this node.
        const uint32_t valid = (1u << ntri) - 1u;
        masks &= valid | (valid << 16);
        uint32_t m = masks & 0xffffu;
        bool first = true;
        while (m) {
            const uint32_t t = (uint32_t)__ffs((int)m) - 1u;
            m &= m - 1u;
            const double q = alpha_with<LAYOUT>(a, nb, __ldg(nb + deg + t), p.x, p.y);
            if (first || q < q_old) q_old = q;
            first = false;
        }
        m = masks >> 16;
        first = true;
        while (m) {
            const uint32_t t = (uint32_t)__ffs((int)m) - 1u;
            m &= m - 1u;
            const double q = alpha_with<LAYOUT>(a, nb, __ldg(nb + deg + t), cx, cy);
            if (first || q < q_new) q_new = q;
            first = false;
        }
    } else {
        for (uint32_t t = 0; t < ntri; ++t) {
            const uint32_t code = __ldg(nb + deg + t);
            const double qo = alpha_with<LAYOUT>(a, nb, code, p.x, p.y);
            const double qn = alpha_with<LAYOUT>(a, nb, code, cx, cy);
            if (t == 0 || qo < q_old) q_old = qo;
            if (t == 0 || qn < q_new) q_new = qn;
        }
    }

    const bool ok = a.strict ? (q_new > q_old) : (q_new >= q_old);
    double2 o = p;
    d2_bits = 0ull;
    moved = ok && (__double_as_longlong(cx) != __double_as_longlong(p.x) ||
                   __double_as_longlong(cy) != __double_as_longlong(p.y));
    if (ok) {
        const double dx = __dsub_rn(cx, p.x), dy = __dsub_rn(cy, p.y);
        const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
        d2_bits = (unsigned long long)__double_as_longlong(d2);
        o = make_double2(cx, cy);
    }
    Coords<LAYOUT>::put(a.out, a.n, i, o);
    if (a.accept) a.accept[i] = ok ? 1 : 0;
    accepted = ok;
}

}  // namespace sls
