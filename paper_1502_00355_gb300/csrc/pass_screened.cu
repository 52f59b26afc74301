// pass_screened.cu -- the fast exact Jacobi pass of Smart Laplacian smoothing.
//
// Same results, bit for bit, as the FP64 pass (Eq. 2 with the accept test of
// Section 3.3.4); what changes is which pipe does which work.  GB300 issues
// about two FP64 operations per SM per clock against ~128 FP32/INT32, so the
// FP64 pipe does only what decides the result's bits, and the rest moves to
// the FP32 and integer pipes:
//
//  1. The neighbour sums (Eq. 2) are the FP64 additions themselves, in the
//     stored summation order.
//  2. The division by the degree is one FP64 multiplication by RN(1/N) and an
//     exact integer remainder that picks the correctly rounded quotient
//     (div_small.cuh), instead of a full division.
//  3. If the centre equals the node's position bit for bit, q_new == q_old
//     exactly and no quality needs evaluating.
//  4. Otherwise alpha of every incident triangle, before and after the move, is
//     evaluated in FP32 in a frame centred on the node, with a rigorous bound
//     on its distance to the exact alpha of the FP64 inputs, wide enough to
//     also cover the FP64 evaluation's own rounding (one bound per side, valid
//     for all of the node's triangles).  The neighbours' local coordinates
//     come from float head/tail splits of the doubles; the centre's offset
//     from one exact FP64 subtraction.  When the intervals of q_new and q_old
//     are disjoint the FP64 decision is known.
//  5. If one triangle alone attains both minima, a second screen takes the
//     sign of alpha(centre) - alpha(node) from a formula in the move itself
//     (no cancellation) and decides all but rounding-level ties.
//  6. What is left goes to a per-warp queue in shared memory and is finished
//     by the exact FP64 update 32 nodes at a time (dense lanes on the narrow
//     FP64 pipe), on the triangles the screen could not rule out.
//
// Coordinates are moved as 64-bit patterns, never held in FP64 registers
// unless they take part in FP64 arithmetic: the compiler copies FP64
// registers with FP64-pipe instructions.
#include <atomic>
#include <cfloat>
#include <mutex>

#include "api_common.h"
#include "div_small.cuh"
#include "kernels.h"
#include "node_exact.cuh"
#include "screen.cuh"

namespace sls {

namespace {

// Degree and triangle limits of the screened path (larger rings take the
// exact path).  13 local-coordinate slots per thread keep seven blocks' shared
// memory within the 164 KB carve-out, which leaves the gathers more L1 than
// 16 slots (1% faster on jittered grids; a Delaunay mesh of random points has
// about 7 nodes in 100,000 above 13).
constexpr int kFastMax = 13;
__constant__ double c_recip[kFastMax + 1];  // RN(1/N)
__constant__ double c_degree[kFastMax + 1]; // N as a double

__device__ __forceinline__ unsigned long long dbits(double v) { return (unsigned long long)__double_as_longlong(v); }
__device__ __forceinline__ double bitsd(unsigned long long b) { return __longlong_as_double((long long)b); }

using namespace scr;

// Screens free or fixed node i of one mesh (Eq. 2 and the accept test of
// Section 3.3.4).  Decided nodes are written and counted here; returns true
// when the node must be finished by the exact path (d filled in).  loc is
// this thread's slice of the shared local-coordinate buffer (stride nthr).
//
// Warp-synchronous: every lane of the warp calls it (have = false for lanes
// without a node).  The neighbour loop runs to the warp's largest degree in
// groups of four, every load of a group issued before its arithmetic; a lane
// past its own degree adds -0 (x + (-0) == x for every double), so each
// lane's sums are its node's, in the stored order.
//
// The accept test is screened with one error bound per side (before and
// after the move) for all of the node's triangles.  The per-triangle bound
//   e * (13.2 |a| + (264.6 + 194 |a|) g),  g = R^2 / s,
// grows with |a| and g, so the side's largest |a|, its largest local
// coordinate R (every vertex of every triangle of that side lies within it)
// and its smallest edge sum s bound every triangle at once.
template <int LAYOUT>
__device__ __forceinline__ bool screen_node(const PassArgs &a, bool have, int64_t i, float2 *loc, int nthr,
                                            Deferred &d, unsigned long long &best, unsigned long long &nacc,
                                            uint32_t &res)
{
    res = 0u;  // decided nodes: bit 0 accepted, bit 1 coordinates changed
    d.node = (int32_t)i;
    d.flags = 0u;
    d.masks = 0u;
    d.pad = 0u;
    d.cx = 0ull;
    d.cy = 0ull;
    uint32_t off = 0u, meta = kMetaFixed;
    if (have) {
        off = __ldg(a.node_off + i);
        meta = __ldg(a.adj + off);
    }
    const bool fixed = (meta & kMetaFixed) != 0u;
    if (have && fixed && a.accept) a.accept[i] = 0;
    const uint32_t deg = fixed ? 0u : meta_degree(meta), ntri = fixed ? 0u : meta_ntri(meta);
    const bool big = !fixed && (deg > (uint32_t)kFastMax || ntri > (uint32_t)kFastMax);
    bool act = have && !fixed && !big;
    const uint32_t *nb = a.adj + off + 1;
    const uint32_t dmax = __reduce_max_sync(0xffffffffu, act ? deg : 0u);

    ulonglong2 pb = make_ulonglong2(0ull, 0ull), v0 = make_ulonglong2(0ull, 0ull);
    if (act) {
        pb = CoordBits<LAYOUT>::get(a.in, a.n, i);
        v0 = CoordBits<LAYOUT>::get(a.in, a.n, __ldg(nb));
    }
    float phx, plx, phy, ply;
    bool ok = head_tail(pb.x, phx, plx) & head_tail(pb.y, phy, ply);
    unsigned long long sxb = v0.x, syb = v0.y;
    float rn = 0.0f, rmin = FLT_MAX;
    {
        float2 L;
        bool ok0;
        local_offset(v0.x, v0.y, phx, plx, phy, ply, L.x, L.y, ok0);
        ok = ok & ok0;
        if (act) loc[0] = L;
        const float rl = fmaxf(fabsf(L.x), fabsf(L.y));
        rn = rl;
        rmin = rl;
    }
    for (uint32_t k0 = 1; k0 < dmax; k0 += 4) {
        uint32_t id[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) id[u] = (act && k0 + u < deg) ? __ldg(nb + k0 + u) : 0u;
        ulonglong2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            v[u] = (act && k0 + u < deg) ? CoordBits<LAYOUT>::get(a.in, a.n, id[u])
                                         : make_ulonglong2(0x8000000000000000ull, 0x8000000000000000ull);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t k = k0 + (uint32_t)u;
            if (k < dmax) {  // warp-uniform
                const bool on = act && k < deg;
                // x + (-0) == x for every x: lanes past their degree add -0
                sxb = dbits(__dadd_rn(bitsd(sxb), bitsd(v[u].x)));
                syb = dbits(__dadd_rn(bitsd(syb), bitsd(v[u].y)));
                float2 L;
                bool okk;
                local_offset(v[u].x, v[u].y, phx, plx, phy, ply, L.x, L.y, okk);
                if (on) loc[k * nthr] = L;
                const float rl = fmaxf(fabsf(L.x), fabsf(L.y));
                rn = on ? fmaxf(rn, rl) : rn;
                rmin = on ? fminf(rmin, rl) : rmin;
                ok = on ? (ok & okk) : ok;
            }
        }
    }
    if (big) return true;  // exact path does it all
    if (!act) return false;
    const double fd = c_degree[deg], y = c_recip[deg];
    const unsigned long long cbx = divs::div_small_bits(sxb, deg, y, fd);
    const unsigned long long cby = divs::div_small_bits(syb, deg, y, fd);
    d.cx = cbx;
    d.cy = cby;
    d.flags = kHasCentre;
    if (cbx == pb.x && cby == pb.y) {
        // the centre is the node itself: q_new == q_old exactly
        const bool acc = !a.strict;
        CoordBits<LAYOUT>::put(a.out, a.n, i, pb);
        if (a.accept) a.accept[i] = acc ? 1 : 0;
        nacc += acc ? 1ull : 0ull;
        res = acc ? 1u : 0u;
        return false;
    }
    if (!ok) return true;
    const double dx = __dsub_rn(bitsd(cbx), bitsd(pb.x)), dy = __dsub_rn(bitsd(cby), bitsd(pb.y));
    const float Cx = trunc_float(dbits(dx)), Cy = trunc_float(dbits(dy));
    const float rC = fmaxf(fabsf(Cx), fabsf(Cy));
    const float M = fmaxf(fabsf(phx), fabsf(phy)) * 1.0001f + fmaxf(rn, rC);
    const float M2 = M * M;
    if (!frame_ok(rmin, fmaxf(rn, rC), M)) return true;
    const float rN = fmaxf(rn, rC);
    float amin_o = FLT_MAX, a2_o = FLT_MAX, amax_o = 0.0f, smin_o = FLT_MAX;
    float amin_n = FLT_MAX, a2_n = FLT_MAX, amax_n = 0.0f, smin_n = FLT_MAX;
    uint32_t arg_o = 0u, arg_n = 0u;
    for (uint32_t t0 = 0; t0 < ntri; t0 += 4) {
        uint32_t c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = t0 + u < ntri ? __ldg(nb + deg + t0 + u) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t t = t0 + (uint32_t)u;
            if (t < ntri) {
                const float2 A = loc[code_first(c[u]) * nthr];
                const float2 B = loc[code_second(c[u]) * nthr];
                const float sk = code_slot(c[u]) == 1u ? -kTwoSqrt3f : kTwoSqrt3f;
                const float ba2 = edge_ba2(A.x, A.y, B.x, B.y);
                {
                    float sv;
                    const float av = screen_alpha(0.0f, 0.0f, A.x, A.y, B.x, B.y, ba2, sk, sv);
                    if (av < amin_o) {
                        a2_o = amin_o;
                        amin_o = av;
                        arg_o = t;
                    } else {
                        a2_o = fminf(a2_o, av);
                    }
                    amax_o = fmaxf(amax_o, fabsf(av));
                    smin_o = fminf(smin_o, sv);
                }
                {
                    float sv;
                    const float av = screen_alpha(Cx, Cy, A.x, A.y, B.x, B.y, ba2, sk, sv);
                    if (av < amin_n) {
                        a2_n = amin_n;
                        amin_n = av;
                        arg_n = t;
                    } else {
                        a2_n = fminf(a2_n, av);
                    }
                    amax_n = fmaxf(amax_n, fabsf(av));
                    smin_n = fminf(smin_n, sv);
                }
            }
        }
    }
    // per side: q (FP64) lies in [amin - b, amin + b]; the minimum is attained
    // by triangle arg alone when every other alpha lies above amin + b + b
    const float go = side_g(rn, smin_o), gn = side_g(rN, smin_n);
    int verdict = 0;
    bool single_o = false, single_n = false;
    const bool bok = bound_ok(smin_o, go, amax_o) & bound_ok(smin_n, gn, amax_n);
    const float bo = side_bound(amax_o, go);
    const float bn = side_bound(amax_n, gn);
    const float minU_o = amin_o + bo, minU_n = amin_n + bn;
    if (bok) {
        const float minL_o = amin_o - bo, minL_n = amin_n - bn;
        verdict = minL_n > minU_o ? 1 : (minU_n < minL_o ? -1 : 0);
        single_o = a2_o - bo > minU_o;
        single_n = a2_n - bn > minU_n;
    }
    if (verdict == 0 && single_o && single_n && arg_o == arg_n) {
        const uint32_t c = __ldg(nb + deg + arg_o);
        const float2 A = loc[code_first(c) * nthr], B = loc[code_second(c) * nthr];
        verdict = diff_screen(A.x, A.y, B.x, B.y, Cx, Cy, code_slot(c) == 1u ? -1.0f : 1.0f, M2);
    }
    if (verdict == 0) {
        // candidates for the exact path: every triangle whose interval
        // reaches below the side's lowest upper end (all of them when the
        // bounds do not hold)
        const uint32_t all = (1u << ntri) - 1u;
        uint32_t mo = bok ? (single_o ? (1u << arg_o) : 0u) : all;
        uint32_t mn = bok ? (single_n ? (1u << arg_n) : 0u) : all;
        if (bok && !(single_o && single_n)) {
            for (uint32_t t = 0; t < ntri; ++t) {
                const uint32_t c = __ldg(nb + deg + t);
                const float2 A = loc[code_first(c) * nthr];
                const float2 B = loc[code_second(c) * nthr];
                const float sk = code_slot(c) == 1u ? -kTwoSqrt3f : kTwoSqrt3f;
                const float ba2 = edge_ba2(A.x, A.y, B.x, B.y);
                float sv;
                if (!single_o && screen_alpha(0.0f, 0.0f, A.x, A.y, B.x, B.y, ba2, sk, sv) - bo <= minU_o)
                    mo |= 1u << t;
                if (!single_n && screen_alpha(Cx, Cy, A.x, A.y, B.x, B.y, ba2, sk, sv) - bn <= minU_n)
                    mn |= 1u << t;
            }
        }
        d.flags |= kMasked;
        d.masks = mo | (mn << 16);
        return true;
    }
    const bool acc = verdict > 0;
    ulonglong2 outp = pb;
    if (acc) {
        const unsigned long long b2 = dbits(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        best = b2 > best ? b2 : best;
        nacc += 1ull;
        outp = make_ulonglong2(cbx, cby);
        res = 3u;  // the centre differs from the node (equal centres return above)
    }
    CoordBits<LAYOUT>::put(a.out, a.n, i, outp);
    if (a.accept) a.accept[i] = acc ? 1 : 0;
    return false;
}

// Finishes one full warp's worth of deferred nodes (lane k takes entry k)
// when the warp's queue holds at least 32, or all remaining entries at the
// end.  Dense lanes keep the narrow FP64 pipe busy without block barriers.
template <int LAYOUT>
__device__ __forceinline__ void drain_queue(const PassArgs &a, Deferred *wq, int &qn, bool all,
                                            unsigned long long &best, unsigned long long &nacc)
{
    const int lane = threadIdx.x & 31;
    while (qn >= 32 || (all && qn > 0)) {
        if (lane < qn) {
            const Deferred e = wq[lane];
            unsigned long long b2;
            bool acc, moved;
            exact_update<LAYOUT>(a, e.node, e.flags, e.masks, e.cx, e.cy, b2, acc, moved);
            best = b2 > best ? b2 : best;
            nacc += acc ? 1ull : 0ull;
            if (a.halo) {  // the node's bits in its tile's masks (written with the tile's other nodes)
                const uint32_t bit = 1u << (e.node & 31);
                if (moved) atomicOr(a.chg_cur + (e.node >> 5), bit);
                if (acc) atomicOr(a.accm + (e.node >> 5), bit);
            }
        }
        const int rest = qn > 32 ? qn - 32 : 0;
        __syncwarp();
        if (lane < rest) wq[lane] = wq[32 + lane];
        __syncwarp();
        qn = rest;
    }
}

// Warp-wide reduction of the statistics into one record (lane 0 writes).
__device__ __forceinline__ void warp_flush_stats(PassStats *st, unsigned long long best,
                                                 unsigned long long nacc, unsigned long long nfb)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, best, o);
        best = m2 > best ? m2 : best;
        nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
        nfb += __shfl_xor_sync(0xffffffffu, nfb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (best) atomicMax(&st->maxd2_bits, best);
        if (nacc) atomicAdd(&st->nacc, nacc);
        if (nfb) atomicAdd(&st->fallbacks, nfb);
    }
}

template <int LAYOUT>
// 128 threads, 7 blocks per SM: 28 warps per SM (72 registers a thread).
__global__ void __launch_bounds__(128, 7) pass_screened_kernel(PassArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nthr = blockDim.x;
    float2 *s_loc = reinterpret_cast<float2 *>(smem_raw);                       // [kFastMax][nthr]
    Deferred *s_q = reinterpret_cast<Deferred *>(s_loc + kFastMax * nthr);      // [64] per warp

    if (pass_is_skipped(a.stats, a.q, a.tol_active, a.thr_bits)) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) a.stats[a.q].executed = 1u;

    unsigned long long best = 0ull, nacc = 0ull, nfb = 0ull;
    unsigned nskip = 0u;  // node updates this warp left as they were (lane 0)
    float2 *loc = s_loc + tid;
    Deferred *wq = s_q + 64 * warp;
    int qn = 0;  // warp-uniform queue length
    // every node in index order, or (a colour class of Form B) the listed
    // nodes or a range of ids
    const int64_t cnt = a.order ? a.norder : (a.ranged ? a.count : a.n);
    const int64_t nwtiles = (cnt + 31) / 32;
    const int64_t wstride = (int64_t)gridDim.x * (nthr >> 5);
    for (int64_t wt = (int64_t)blockIdx.x * (nthr >> 5) + warp; wt < nwtiles; wt += wstride) {
        if (a.skip) {
            // the tile's inputs: its own nodes and every neighbour, by tile
            const uint2 h = lane < kHaloEntries ? __ldg(a.halo + wt * kHaloEntries + lane) : make_uint2(0u, 0u);
            const bool never = __shfl_sync(0xffffffffu, h.x, 0) == kHaloNever;
            const uint32_t c = h.y != 0u ? __ldg(a.chg_prev + h.x) & h.y : 0u;
            if (!__any_sync(0xffffffffu, c != 0u) && !never) {
                // all unchanged: the same inputs as in the previous pass, so the
                // same results, which `out` and the masks already hold
                if (lane == 0) {
                    a.chg_cur[wt] = 0u;
                    nacc += (unsigned long long)__popc(a.accm[wt]);
                    nskip += (unsigned)(a.n - wt * 32 < 32 ? a.n - wt * 32 : 32);
                }
                continue;
            }
        }
        const int64_t j = wt * 32 + lane;
        Deferred d;
        const bool have = j < cnt;
        uint32_t res;
        const bool defer = screen_node<LAYOUT>(a, have, have ? (a.order ? (int64_t)__ldg(a.order + j) : a.first + j) : 0,
                                               loc, nthr, d, best, nacc, res);
        const unsigned m = __ballot_sync(0xffffffffu, defer);
        if (a.halo) {  // before any drain: deferred nodes add their bits there
            const unsigned cb = __ballot_sync(0xffffffffu, (res & 2u) != 0u);
            const unsigned ab = __ballot_sync(0xffffffffu, (res & 1u) != 0u);
            if (lane == 0) {
                a.chg_cur[wt] = cb;
                a.accm[wt] = ab;
            }
        }
        if (defer) wq[qn + __popc(m & ((1u << lane) - 1u))] = d;
        qn += __popc(m);
        nfb += defer ? 1ull : 0ull;
        if (qn >= 32) {  // warp-uniform; entries written by other lanes must be visible
            __syncwarp();
            drain_queue<LAYOUT>(a, wq, qn, false, best, nacc);
        }
    }
    __syncwarp();
    drain_queue<LAYOUT>(a, wq, qn, true, best, nacc);
    if (nskip) atomicAdd(&a.stats[a.q].nodes_skipped, nskip);
    block_reduce_stats(a.stats + a.q, best, nacc, nfb);
}

// ---- batched / served form: many meshes, one launch per round -----------
// Work is a list of warp tasks (32 consecutive nodes of one job).  With
// chunk > 0 the warps take chunks of `chunk` consecutive tasks in a grid
// stride (warp w: chunks w, w + W, w + 2W, ...), so that at any moment they
// work on a window of neighbouring tasks and share its gathers in L1 and L2;
// with chunk < 0 they claim chunks of -chunk tasks in list order from the
// round's counter (*claim, zero at the launch), which keeps that window and
// lets a warp that drew cheap tasks take more; chunk = 0 gives each warp one
// contiguous share of the list.  A job takes part in
// round r as its pass q = r - base_round while q < max_iter and its
// tolerance is not met.  The deferred queue is drained and the statistics
// flushed whenever the warp moves to another job, so every record gets
// exactly its own job's counts.
template <int LAYOUT>
__global__ void __launch_bounds__(128, 6) batch_pass_kernel(const JobDesc *__restrict__ jobs,
                                                          const WarpTask *__restrict__ tasks, int64_t ntasks,
                                                          int round, int64_t chunk,
                                                          unsigned long long *claim)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nthr = blockDim.x;
    float2 *s_loc = reinterpret_cast<float2 *>(smem_raw);
    Deferred *s_q = reinterpret_cast<Deferred *>(s_loc + kFastMax * nthr);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *loc = s_loc + tid;
    Deferred *wq = s_q + 64 * warp;

    const int64_t nwarps = (int64_t)gridDim.x * (nthr >> 5);
    const int64_t gw = (int64_t)blockIdx.x * (nthr >> 5) + warp;
    const bool dynamic = chunk < 0;
    const int64_t per = chunk > 0 ? chunk : (dynamic ? -chunk : (ntasks + nwarps - 1) / nwarps);
    const int64_t cstride = chunk > 0 ? nwarps * chunk : ntasks;  // one share per warp when chunk == 0
    auto claim_next = [&]() -> int64_t {
        unsigned long long v = 0ull;
        if (lane == 0) v = atomicAdd(claim, (unsigned long long)per);
        return (int64_t)__shfl_sync(0xffffffffu, v, 0);
    };
    int64_t c0 = dynamic ? claim_next() : gw * per;  // first task of the current chunk
    int64_t t = c0;

    int cur_job = -1;
    bool active = false;
    PassArgs a{};
    unsigned long long best = 0ull, nacc = 0ull, nfb = 0ull;
    int qn = 0;
    for (;;) {
        if (t >= c0 + per || t >= ntasks) {  // next chunk of this warp
            c0 = dynamic ? (c0 < ntasks ? claim_next() : c0) : c0 + cstride;
            t = c0;
        }
        const bool more = t < ntasks && c0 < ntasks;
        const int job = more ? tasks[t].job : -2;
        if (job != cur_job) {
            if (cur_job >= 0 && active) {
                __syncwarp();
                drain_queue<LAYOUT>(a, wq, qn, true, best, nacc);
                warp_flush_stats(a.stats + a.q, best, nacc, nfb);
            }
            best = nacc = nfb = 0ull;
            cur_job = job;
            if (job < 0) break;
            const JobDesc *J = jobs + job;
            const int q = round - J->base_round;
            PassStats *st = J->stats;
            const int tol_active = J->tol_active;
            const unsigned long long thr_bits = J->thr_bits;
            active = q >= 0 && q < J->max_iter && !pass_is_skipped(st, q, tol_active, thr_bits);
            if (active) {
                double *x0 = J->xy[0], *x1 = J->xy[1];
                const bool odd = ((J->cur0 + q) & 1) != 0;
                a.in = odd ? x1 : x0;
                a.out = odd ? x0 : x1;
                a.node_off = J->node_off;
                a.adj = J->adj;
                a.n = J->n;
                a.order = nullptr;
                a.norder = 0;
                a.stats = st;
                a.q = q;
                a.strict = J->strict;
                a.tol_active = tol_active;
                a.thr_bits = thr_bits;
                a.accept = J->accept;
            }
        }
        if (!active) {
            ++t;
            continue;
        }
        const int64_t first = tasks[t].first;
        ++t;
        if (first == 0 && lane == 0) a.stats[a.q].executed = 1u;
        const int64_t i = first + lane;
        Deferred d;
        uint32_t res;
        const bool defer = screen_node<LAYOUT>(a, i < a.n, i < a.n ? i : 0, loc, nthr, d, best, nacc, res);
        const unsigned m = __ballot_sync(0xffffffffu, defer);
        if (defer) wq[qn + __popc(m & ((1u << lane) - 1u))] = d;
        qn += __popc(m);
        nfb += defer ? 1ull : 0ull;
        if (qn >= 32) {
            __syncwarp();
            drain_queue<LAYOUT>(a, wq, qn, false, best, nacc);
        }
    }
}

// Constant memory and function attributes belong to a context: they are set
// up once per device and context, with that device current (a context made
// after cudaDeviceReset is set up again).
constexpr int kMaxDevices = 64;
std::atomic<unsigned long long> g_consts_ctx[kMaxDevices] = {};
std::mutex g_consts_mu;

cudaError_t ensure_constants()
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long id = current_context_id();
    const unsigned long long key = id ? id : ~0ull;  // ~0: the context is not known yet
    if (g_consts_ctx[dev].load(std::memory_order_acquire) == key) return cudaSuccess;
    std::lock_guard<std::mutex> lock(g_consts_mu);
    if (g_consts_ctx[dev].load(std::memory_order_relaxed) == key) return cudaSuccess;
    double r[kFastMax + 1];
    double dg[kFastMax + 1];
    r[0] = 0.0;
    dg[0] = 0.0;
    for (int k = 1; k <= kFastMax; ++k) {
        r[k] = 1.0 / (double)k;
        dg[k] = (double)k;
    }
    e = cudaMemcpyToSymbol(c_recip, r, sizeof r);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_degree, dg, sizeof dg);
    if (e != cudaSuccess) return e;
    const void *fns[4] = {(const void *)pass_screened_kernel<0>, (const void *)pass_screened_kernel<1>,
                          (const void *)batch_pass_kernel<0>, (const void *)batch_pass_kernel<1>};
    for (const void *f : fns) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
    }
    g_consts_ctx[dev].store(key, std::memory_order_release);
    return cudaSuccess;
}

}  // namespace

size_t screened_smem_bytes(int block)
{
    return (size_t)block * (kFastMax * sizeof(float2) + 2 * sizeof(Deferred));  // 64 entries per warp
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

cudaError_t launch_batch_pass(const JobDesc *jobs, const WarpTask *tasks, int64_t ntasks, int round,
                              int layout, int block, int grid, cudaStream_t s, int64_t chunk,
                              unsigned long long *claim)
{
    cudaError_t e = ensure_constants();
    if (e != cudaSuccess) return e;
    if (ntasks <= 0) return cudaSuccess;
    if (chunk < 0 && !claim) return cudaErrorInvalidValue;
    const size_t smem = screened_smem_bytes(block);
    if (layout == 0) batch_pass_kernel<0><<<grid, block, smem, s>>>(jobs, tasks, ntasks, round, chunk, claim);
    else batch_pass_kernel<1><<<grid, block, smem, s>>>(jobs, tasks, ntasks, round, chunk, claim);
    return cudaGetLastError();
}

namespace {

__global__ void gather_round_kernel(const JobDesc *__restrict__ jobs, int na, int round, PassStats *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= na) return;
    const JobDesc &J = jobs[j];
    int q = round - J.base_round;
    const int last = J.max_iter > 1 ? J.max_iter - 1 : 0;
    q = q < last ? q : last;
    out[j] = J.stats[q];
}

// The warp tasks of na jobs: job j's 32-node tasks at task_off[j] onwards.
__global__ void expand_tasks_kernel(const JobDesc *__restrict__ jobs, const int64_t *__restrict__ task_off, int na,
                                    WarpTask *__restrict__ tasks)
{
    for (int j = blockIdx.x; j < na; j += gridDim.x) {
        const int64_t n = jobs[j].n, t0 = task_off[j];
        for (int64_t f = (int64_t)threadIdx.x * 32; f < n; f += (int64_t)blockDim.x * 32)
            tasks[t0 + f / 32] = WarpTask{j, (int32_t)f};
    }
}

}  // namespace

cudaError_t launch_expand_tasks(const JobDesc *jobs, const int64_t *task_off, int na, WarpTask *tasks,
                                cudaStream_t s)
{
    if (na <= 0) return cudaSuccess;
    expand_tasks_kernel<<<na < 4096 ? na : 4096, 256, 0, s>>>(jobs, task_off, na, tasks);
    return cudaGetLastError();
}

cudaError_t launch_gather_round(const JobDesc *jobs, int na, int round, PassStats *out, cudaStream_t s)
{
    if (na <= 0) return cudaSuccess;
    gather_round_kernel<<<(na + 127) / 128, 128, 0, s>>>(jobs, na, round, out);
    return cudaGetLastError();
}

int batch_pass_occupancy(int layout, int block)
{
    if (ensure_constants() != cudaSuccess) return 1;
    int nb = 0;
    const size_t smem = screened_smem_bytes(block);
    if (layout == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_pass_kernel<0>, block, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_pass_kernel<1>, block, smem);
    return nb > 0 ? nb : 1;
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
