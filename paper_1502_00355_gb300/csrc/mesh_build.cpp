// mesh_build.cpp -- host-side mesh validation and adjacency construction.
//
// Section 3.3.2 of the paper finds, for every vertex, its neighbouring
// vertices (the other two vertices of each incident triangle) and its
// incident triangles; the paper runs this on a single GPU thread because of
// the write dependencies.  Here it is a two-phase host build: a counting sort
// of the 3m incidences, each carrying the triangle's other two vertices and
// the node's slot (so the per-node passes read their own records in order
// instead of gathering triangles), then an independent per-node pass (run on
// all host cores) that de-duplicates the neighbours, counts how many
// triangles share each edge, and orders the neighbours for summation.
//
// Section 3.3.3 marks a vertex as internal when each of its neighbours has
// been recorded twice; a neighbour recorded once means a boundary edge, so
// the vertex is fixed.  A neighbour recorded three or more times means a
// non-manifold edge, which is rejected.
//
// Summation order (the paper does not give one): ascending x of the creation
// coordinates, then ascending y, then ascending node id.  It depends on
// geometry only, so renumbering the nodes does not change any result.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "internal.h"

namespace sls {

namespace {

struct Range {
    int64_t lo, hi;
};

template <class F>
void parallel_for_nodes(int64_t n, int threads, F &&body)
{
    if (threads <= 1 || n < 4096) {
        body(Range{0, n});
        return;
    }
    std::vector<std::thread> pool;
    int64_t chunk = (n + threads - 1) / threads;
    for (int t = 0; t < threads; ++t) {
        int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
        if (lo >= hi) break;
        pool.emplace_back([&body, lo, hi] { body(Range{lo, hi}); });
    }
    for (auto &th : pool) th.join();
}

}  // namespace

double bbox_diagonal(double xmin, double xmax, double ymin, double ymax)
{
    const double wx = xmax - xmin, wy = ymax - ymin;
    const double wx2 = wx * wx, wy2 = wy * wy;
    return std::sqrt(wx2 + wy2);
}

sls_status build_host_mesh(const double *xy, int64_t n, const int32_t *tri, int64_t m,
                           const uint8_t *boundary, HostMesh &out, int threads)
{
    if (!xy || !tri) return fail(SLS_ERR_INVALID, "xy and tri must not be NULL");
    if (n < 3) return fail(SLS_ERR_INVALID, "a mesh needs at least 3 nodes");
    if (m < 1) return fail(SLS_ERR_INVALID, "a mesh needs at least 1 triangle");
    if (n >= (int64_t(1) << 31) || m >= (int64_t(1) << 31))
        return fail(SLS_ERR_INVALID, "n and m must be below 2^31");
    if (threads <= 0) threads = (int)std::min(32u, std::max(1u, std::thread::hardware_concurrency()));

    for (int64_t k = 0; k < 2 * n; ++k)
        if (!std::isfinite(xy[k]))
            return fail(SLS_ERR_INVALID, "coordinate " + std::to_string(k) + " is not finite");
    for (int64_t t = 0; t < m; ++t) {
        int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n)
            return fail(SLS_ERR_INVALID, "triangle " + std::to_string(t) + " has a vertex id out of range");
        if (a == b || a == c || b == c)
            return fail(SLS_ERR_INVALID, "triangle " + std::to_string(t) + " repeats a vertex");
    }

    // Incidences sorted by vertex (counting sort keeps ascending triangle ids).
    std::vector<int64_t> inc_ptr(n + 1, 0);
    for (int64_t k = 0; k < 3 * m; ++k) inc_ptr[tri[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
    // each incidence keeps the other two vertices (stored order) and the slot
    struct Inc {
        int32_t a, b;
        uint32_t slot;
    };
    std::vector<Inc> inc(3 * m);
    {
        std::vector<int64_t> cursor(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t t = 0; t < m; ++t) {
            const int32_t v0 = tri[3 * t], v1 = tri[3 * t + 1], v2 = tri[3 * t + 2];
            inc[cursor[v0]++] = Inc{v1, v2, 0u};
            inc[cursor[v1]++] = Inc{v0, v2, 1u};
            inc[cursor[v2]++] = Inc{v0, v1, 2u};
        }
    }

    // Phase 1: per node, the distinct neighbours in summation order, stored in
    // the node's own slice [2*inc_ptr[i], 2*inc_ptr[i+1]) of a scratch array.
    std::vector<int32_t> nb(6 * m);
    std::vector<uint32_t> deg(n), ntri(n);
    std::vector<uint8_t> fixed(n);
    std::atomic<int> bad{0};
    auto phase1 = [&](Range r) {
        std::vector<int32_t> rec;
        int nonmanifold = 0;
        for (int64_t i = r.lo; i < r.hi; ++i) {
            rec.clear();
            for (int64_t k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
                rec.push_back(inc[k].a);
                rec.push_back(inc[k].b);
            }
            std::sort(rec.begin(), rec.end());
            int32_t *dst = nb.data() + 2 * inc_ptr[i];
            uint32_t d = 0;
            bool open_edge = rec.empty();
            for (size_t k = 0; k < rec.size();) {
                size_t e = k;
                while (e < rec.size() && rec[e] == rec[k]) ++e;
                size_t times = e - k;
                if (times == 1) open_edge = true;
                if (times > 2) nonmanifold = 1;
                dst[d++] = rec[k];
                k = e;
            }
            std::sort(dst, dst + d, [xy](int32_t p, int32_t q) {
                double xp = xy[2 * (int64_t)p], xq = xy[2 * (int64_t)q];
                if (xp < xq) return true;
                if (xq < xp) return false;
                double yp = xy[2 * (int64_t)p + 1], yq = xy[2 * (int64_t)q + 1];
                if (yp < yq) return true;
                if (yq < yp) return false;
                return p < q;
            });
            deg[i] = d;
            ntri[i] = (uint32_t)(inc_ptr[i + 1] - inc_ptr[i]);
            bool fx = boundary ? (boundary[i] != 0 || rec.empty()) : open_edge;
            fixed[i] = fx ? 1 : 0;
            if (!fx && (d > (uint32_t)MAX_DEGREE || ntri[i] > (uint32_t)MAX_DEGREE)) nonmanifold |= 2;
        }
        if (nonmanifold) bad.fetch_or(nonmanifold);
    };
    parallel_for_nodes(n, threads, phase1);
    int any_bad = bad.load();
    if (any_bad & 1) return fail(SLS_ERR_NONMANIFOLD, "an edge is shared by more than two triangles");
    if (any_bad & 2) return fail(SLS_ERR_INVALID, "a free node has more than 32767 neighbours or triangles");

    // Offsets of the per-node word groups.
    out.node_off.assign(n + 1, 0);
    uint64_t words = 0;
    int64_t n_free = 0;
    for (int64_t i = 0; i < n; ++i) {
        out.node_off[i] = (uint32_t)words;
        words += fixed[i] ? 1 : 1 + (uint64_t)deg[i] + ntri[i];
        n_free += fixed[i] ? 0 : 1;
        if (words >= (uint64_t(1) << 32)) return fail(SLS_ERR_INVALID, "adjacency exceeds 2^32 words");
    }
    out.node_off[n] = (uint32_t)words;
    out.adj.assign(words, 0);

    // Phase 2: write the words; triangle codes refer to neighbour positions.
    auto phase2 = [&](Range r) {
        for (int64_t i = r.lo; i < r.hi; ++i) {
            uint32_t *w = out.adj.data() + out.node_off[i];
            if (fixed[i]) {
                w[0] = meta_word(true, 0, 0);
                continue;
            }
            const int32_t *list = nb.data() + 2 * inc_ptr[i];
            uint32_t d = deg[i];
            w[0] = meta_word(false, d, ntri[i]);
            for (uint32_t k = 0; k < d; ++k) w[1 + k] = (uint32_t)list[k];
            uint32_t *codes = w + 1 + d;
            uint32_t c = 0;
            for (int64_t k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
                const Inc &r = inc[k];
                uint32_t pa = 0, pb = 0;
                while (list[pa] != r.a) ++pa;
                while (list[pb] != r.b) ++pb;
                codes[c++] = tri_code(r.slot, pa, pb);
            }
        }
    };
    parallel_for_nodes(n, threads, phase2);

    // D: bounding-box diagonal of the input coordinates.
    double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
    for (int64_t i = 1; i < n; ++i) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        xmin = x < xmin ? x : xmin;
        xmax = x > xmax ? x : xmax;
        ymin = y < ymin ? y : ymin;
        ymax = y > ymax ? y : ymax;
    }
    out.diag = bbox_diagonal(xmin, xmax, ymin, ymax);

    out.n = n;
    out.m = m;
    out.n_free = n_free;
    out.fixed.swap(fixed);
    return SLS_OK;
}

}  // namespace sls
