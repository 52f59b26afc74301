// mesh_build_gpu.cu -- the adjacency build of sls_mesh_create on the device.
//
// Same output, word for word, as the host build in mesh_build.cpp (Section
// 3.3.2: neighbours and incident triangles; Section 3.3.3: constraints), with
// the work spread over one thread per triangle or per node instead of the
// paper's single GPU thread:
//   1. validate triangles and coordinates;
//   2. count the incidences of every node, exclusive scan;
//   3. scatter (node, triangle) incidences;
//   4. per node: sort its incident triangles, collect the other vertices of
//      each, sort and de-duplicate them while counting how many triangles
//      share each edge (1 = boundary edge, > 2 = non-manifold), order the
//      neighbours for summation (ascending x, y, id) and size its word group;
//   5. exclusive scan of the word counts -> node offsets;
//   6. per node: write the meta word, the neighbours and the triangle codes;
//   7. bounding box and free-node count.
// Nodes with more than kMaxInc incident triangles are left to the host build
// (the whole mesh then takes the host path).
#include <cstring>
#include <vector>

#include "api_common.h"
#include "kernels.h"

namespace sls {

namespace {

constexpr int kMaxInc = 32;  // incident triangles per node handled on the device

enum : unsigned { kErrRange = 1u, kErrRepeat = 2u, kErrFinite = 4u, kErrManifold = 8u, kErrTooMany = 16u };

__global__ void validate_tri_kernel(const int32_t *__restrict__ tri, int64_t m, int64_t n, unsigned *flags,
                                    unsigned long long *first)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += stride) {
        const int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        const bool range = a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n;
        const bool rep = a == b || a == c || b == c;
        if (range || rep) {
            atomicOr(flags, range ? kErrRange : kErrRepeat);
            // the first bad triangle; at equal index the range error comes first
            atomicMin(first, (unsigned long long)t * 2ull + (range ? 0ull : 1ull));
        }
    }
}

__global__ void validate_xy_kernel(const unsigned long long *__restrict__ xy, int64_t n2, unsigned *flags,
                                   unsigned long long *first)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride) {
        if (((xy[k] >> 52) & 0x7ffull) == 0x7ffull) {
            atomicOr(flags, kErrFinite);
            atomicMin(first, (unsigned long long)k);
        }
    }
}

__global__ void count_kernel(const int32_t *__restrict__ tri, int64_t m3, unsigned *cnt)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m3; k += stride)
        atomicAdd(cnt + tri[k], 1u);
}

__global__ void scatter_kernel(const int32_t *__restrict__ tri, int64_t m3, const unsigned *__restrict__ ptr,
                               unsigned *cursor, int32_t *inc)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m3; k += stride) {
        const int32_t v = tri[k];
        const unsigned slot = atomicAdd(cursor + v, 1u);
        inc[ptr[v] + slot] = (int32_t)(k / 3);
    }
}

// Ascending (x, y, id) with the comparisons of the host build.
__device__ __forceinline__ bool canon_less(double xa, double ya, int32_t a, double xb, double yb, int32_t b)
{
    if (xa < xb) return true;
    if (xb < xa) return false;
    if (ya < yb) return true;
    if (yb < ya) return false;
    return a < b;
}

__global__ void node_pass1_kernel(int64_t n, const double2 *__restrict__ xy, const int32_t *__restrict__ tri,
                                  const unsigned *__restrict__ ptr, int32_t *inc, const uint8_t *boundary,
                                  int32_t *nbtmp, unsigned *words, uint8_t *fixed_out, unsigned *deg_out,
                                  unsigned *flags)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned s = ptr[i], e = ptr[i + 1], nt = e - s;
        if (nt > (unsigned)kMaxInc) {
            atomicOr(flags, kErrTooMany);
            words[i] = 1u;
            fixed_out[i] = 1;
            deg_out[i] = 0u;
            continue;
        }
        int32_t tl[kMaxInc];
        for (unsigned k = 0; k < nt; ++k) {
            const int32_t t = inc[s + k];
            unsigned j = k;
            while (j > 0 && tl[j - 1] > t) {
                tl[j] = tl[j - 1];
                --j;
            }
            tl[j] = t;
        }
        for (unsigned k = 0; k < nt; ++k) inc[s + k] = tl[k];
        // the other two vertices of every incident triangle, sorted by id
        int32_t rec[2 * kMaxInc];
        unsigned r = 0;
        for (unsigned k = 0; k < nt; ++k) {
            for (int c = 0; c < 3; ++c) {
                const int32_t v = tri[3 * (int64_t)tl[k] + c];
                if (v == (int32_t)i) continue;
                unsigned j = r++;
                while (j > 0 && rec[j - 1] > v) {
                    rec[j] = rec[j - 1];
                    --j;
                }
                rec[j] = v;
            }
        }
        bool open_edge = r == 0;
        unsigned deg = 0;
        int32_t uq[2 * kMaxInc];
        for (unsigned k = 0; k < r;) {
            unsigned f = k;
            while (f < r && rec[f] == rec[k]) ++f;
            const unsigned times = f - k;
            if (times == 1u) open_edge = true;
            if (times > 2u) atomicOr(flags, kErrManifold);
            uq[deg++] = rec[k];
            k = f;
        }
        // summation order: ascending (x, y, id) of the creation coordinates
        double ux[2 * kMaxInc], uy[2 * kMaxInc];
        for (unsigned k = 0; k < deg; ++k) {
            const double2 p = xy[uq[k]];
            const int32_t id = uq[k];
            unsigned j = k;
            while (j > 0 && canon_less(p.x, p.y, id, ux[j - 1], uy[j - 1], uq[j - 1])) {
                ux[j] = ux[j - 1];
                uy[j] = uy[j - 1];
                uq[j] = uq[j - 1];
                --j;
            }
            ux[j] = p.x;
            uy[j] = p.y;
            uq[j] = id;
        }
        for (unsigned k = 0; k < deg; ++k) nbtmp[2ull * s + k] = uq[k];
        const bool fx = boundary ? (boundary[i] != 0 || r == 0) : open_edge;
        fixed_out[i] = fx ? 1 : 0;
        deg_out[i] = deg;
        words[i] = fx ? 1u : 1u + deg + nt;
    }
}

__global__ void node_pass2_kernel(int64_t n, const int32_t *__restrict__ tri, const unsigned *__restrict__ ptr,
                                  const int32_t *__restrict__ inc, const int32_t *__restrict__ nbtmp,
                                  const unsigned *__restrict__ deg_in, const uint8_t *__restrict__ fixed_in,
                                  const uint32_t *__restrict__ node_off, uint32_t *adj)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t *w = adj + node_off[i];
        if (fixed_in[i]) {
            w[0] = 0x80000000u;
            continue;
        }
        const unsigned s = ptr[i], nt = ptr[i + 1] - s, deg = deg_in[i];
        w[0] = (nt << 16) | deg;
        const int32_t *list = nbtmp + 2ull * s;
        for (unsigned k = 0; k < deg; ++k) w[1 + k] = (uint32_t)list[k];
        for (unsigned k = 0; k < nt; ++k) {
            const int32_t *v = tri + 3 * (int64_t)inc[s + k];
            uint32_t slot = 0, pos[2] = {0u, 0u}, np = 0;
            for (int c = 0; c < 3; ++c) {
                if (v[c] == (int32_t)i) {
                    slot = (uint32_t)c;
                    continue;
                }
                uint32_t p = 0;
                while (p + 1 < deg && list[p] != v[c]) ++p;
                pos[np++] = p;
            }
            w[1 + deg + k] = (slot << 30) | (pos[0] << 15) | pos[1];
        }
    }
}

// Order-preserving 64-bit keys of finite doubles, for min / max with atomics.
__device__ __forceinline__ unsigned long long okey(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__global__ void bbox_kernel(const double2 *__restrict__ xy, int64_t n, const uint8_t *__restrict__ fixed,
                            unsigned long long *keys /* xmin, ymin, xmax, ymax */, unsigned long long *nfree)
{
    unsigned long long lo_x = ~0ull, lo_y = ~0ull, hi_x = 0ull, hi_y = 0ull, free_cnt = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 p = xy[i];
        const unsigned long long kx = okey(p.x), ky = okey(p.y);
        lo_x = kx < lo_x ? kx : lo_x;
        lo_y = ky < lo_y ? ky : lo_y;
        hi_x = kx > hi_x ? kx : hi_x;
        hi_y = ky > hi_y ? ky : hi_y;
        free_cnt += fixed[i] ? 0ull : 1ull;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t;
        t = __shfl_xor_sync(0xffffffffu, lo_x, o); lo_x = t < lo_x ? t : lo_x;
        t = __shfl_xor_sync(0xffffffffu, lo_y, o); lo_y = t < lo_y ? t : lo_y;
        t = __shfl_xor_sync(0xffffffffu, hi_x, o); hi_x = t > hi_x ? t : hi_x;
        t = __shfl_xor_sync(0xffffffffu, hi_y, o); hi_y = t > hi_y ? t : hi_y;
        free_cnt += __shfl_xor_sync(0xffffffffu, free_cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(keys + 0, lo_x);
        atomicMin(keys + 1, lo_y);
        atomicMax(keys + 2, hi_x);
        atomicMax(keys + 3, hi_y);
        atomicAdd(nfree, free_cnt);
    }
}

// Exclusive scan of cnt[0..len) into out[0..len] (out[len] = total), in three
// steps: per-block sums, a single-block scan of those sums, per-block scans.
constexpr int kScanBlock = 1024;
constexpr int kScanItems = 4;  // per thread

__global__ void scan_sums_kernel(const unsigned *__restrict__ in, int64_t len, unsigned long long *sums)
{
    __shared__ unsigned long long s[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems;
    unsigned long long acc = 0ull;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t j = base + (int64_t)k * kScanBlock + threadIdx.x;
        if (j < len) acc += in[j];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = s[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = acc;
    }
}

__global__ void scan_offsets_kernel(unsigned long long *sums, int64_t nblocks)
{
    // one thread: the block count is small (len / 4096)
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    unsigned long long run = 0ull;
    for (int64_t b = 0; b < nblocks; ++b) {
        const unsigned long long v = sums[b];
        sums[b] = run;
        run += v;
    }
    sums[nblocks] = run;
}

__global__ void scan_final_kernel(const unsigned *__restrict__ in, int64_t len,
                                  const unsigned long long *__restrict__ offs, uint32_t *out)
{
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems;
    if (threadIdx.x == 0) carry = offs[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t j = base + (int64_t)k * kScanBlock + threadIdx.x;
        const unsigned long long v = j < len ? in[j] : 0ull;
        unsigned long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long t = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;  // inclusive over warps
        }
        __syncthreads();
        const unsigned long long before = carry + (warp ? warp_tot[warp - 1] : 0ull) + x - v;
        if (j < len) out[j] = (uint32_t)before;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[len] = (uint32_t)offs[gridDim.x];
}

// A device buffer of the build, from the library's pool on stream s (memory
// comes and goes in stream order, so no call waits for the whole device).
// `async` tells the build whether it may synchronise s (a single mesh's
// build does; the served form builds jobs while rounds run).
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() { pool_free(p, s); }
};

struct Alloc {
    bool async;
    cudaStream_t s;
};

cudaError_t raw_alloc(const Alloc &a, void **p, size_t bytes) { return pool_alloc(p, bytes, a.s); }

#define GB_TRY(expr, what)                                  \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

template <class T>
sls_status dalloc(DevBuf &b, size_t count, T **out, const char *what, const Alloc &a)
{
    b.s = a.s;
    cudaError_t e = raw_alloc(a, &b.p, sizeof(T) * (count > 0 ? count : 1));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SLS_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    *out = static_cast<T *>(b.p);
    return SLS_OK;
}

// scan of len uint32 values into len+1 offsets; total returned (uint64)
sls_status scan_u32(const unsigned *in, int64_t len, uint32_t *out, unsigned long long *total, cudaStream_t s,
                    bool async = false)
{
    const int64_t per_block = (int64_t)kScanBlock * kScanItems;
    const int64_t nblocks = (len + per_block - 1) / per_block;
    DevBuf sb;
    unsigned long long *sums = nullptr;
    sls_status st = dalloc(sb, (size_t)nblocks + 1, &sums, "scan", Alloc{async, s});
    if (st != SLS_OK) return st;
    if (nblocks > 0) {
        scan_sums_kernel<<<(unsigned)nblocks, kScanBlock, 0, s>>>(in, len, sums);
        scan_offsets_kernel<<<1, 1, 0, s>>>(sums, nblocks);
        scan_final_kernel<<<(unsigned)nblocks, kScanBlock, 0, s>>>(in, len, sums, out);
        GB_TRY(cudaGetLastError(), "scan");
        GB_TRY(cudaMemcpyAsync(total, sums + nblocks, sizeof *total, cudaMemcpyDeviceToHost, s), "scan total");
    } else {
        GB_TRY(cudaMemsetAsync(out, 0, sizeof(uint32_t), s), "scan");
        *total = 0ull;
    }
    GB_TRY(cudaStreamSynchronize(s), "scan");
    return SLS_OK;
}

// One block of kOrderTile threads per tile: the number of free nodes (of
// colour c, when colour is given).
__global__ void __launch_bounds__(kOrderTile) order_count_kernel(const uint32_t *__restrict__ node_off,
                                                                  const uint32_t *__restrict__ adj, int64_t n,
                                                                  const int32_t *__restrict__ colour, int32_t c,
                                                                  unsigned *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * kOrderTile + threadIdx.x;
    const bool fr = i < n && !(adj[node_off[i]] & 0x80000000u) && (!colour || colour[i] == c);
    const int k = __syncthreads_count(fr);
    if (threadIdx.x == 0) cnt[blockIdx.x] = (unsigned)k;
}

// One block of kOrderTile threads per tile: the tile's free nodes of the
// class in id order (a bitonic sort of the members' ids in shared memory,
// non-members sorting last), written at the tile's offset.
__global__ void __launch_bounds__(kOrderTile) order_sort_kernel(const uint32_t *__restrict__ node_off,
                                                                 const uint32_t *__restrict__ adj, int64_t n,
                                                                 const int32_t *__restrict__ colour, int32_t c,
                                                                 const uint32_t *__restrict__ tile_off,
                                                                 uint32_t *order)
{
    __shared__ uint32_t key[kOrderTile];
    const unsigned tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kOrderTile + tid;
    uint32_t k = 0xffffffffu;  // fixed nodes and the tail sort last
    if (i < n) {
        const uint32_t meta = adj[node_off[i]];
        if (!(meta & 0x80000000u) && (!colour || colour[i] == c))
            k = tid;
    }
    key[tid] = k;
    __syncthreads();
    for (unsigned size = 2; size <= (unsigned)kOrderTile; size <<= 1) {
        for (unsigned stride = size >> 1; stride > 0; stride >>= 1) {
            const unsigned j = tid ^ stride;
            if (j > tid) {
                const uint32_t a = key[tid], b = key[j];
                const bool up = (tid & size) == 0;
                if ((a > b) == up) {
                    key[tid] = b;
                    key[j] = a;
                }
            }
            __syncthreads();
        }
    }
    const uint32_t nf = tile_off[blockIdx.x + 1] - tile_off[blockIdx.x];
    if (tid < nf) order[tile_off[blockIdx.x] + tid] = (uint32_t)(blockIdx.x * kOrderTile) + (key[tid] & 1023u);
}

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the colouring priorities.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Initial colouring state: -2 fixed, -1 free and uncoloured.
__global__ void colour_init_kernel(const uint32_t *__restrict__ node_off, const uint32_t *__restrict__ adj,
                                   int64_t n, int32_t *colour)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        colour[i] = (adj[node_off[i]] & 0x80000000u) ? -2 : -1;
}

// One Jones-Plassmann round.  cur is the state at the start of the round,
// next a copy of it that receives the winners' colours: an uncoloured free
// node wins when its (priority, index) exceeds that of every uncoloured free
// neighbour, and takes the smallest colour no neighbour holds.  Winners are
// never neighbours, so the round's result does not depend on thread order.
__global__ void colour_round_kernel(const uint32_t *__restrict__ node_off, const uint32_t *__restrict__ adj,
                                    int64_t n, unsigned long long seed, const int32_t *__restrict__ cur,
                                    int32_t *next, unsigned long long *left, unsigned *flags)
{
    unsigned long long cnt = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (cur[i] != -1) continue;
        const uint32_t *w = adj + node_off[i];
        const uint32_t deg = w[0] & 0xffffu;
        const unsigned long long pi = splitmix64(seed + (unsigned long long)i);
        bool win = true;
        unsigned long long used = 0ull;
        for (uint32_t k = 0; k < deg; ++k) {
            const uint32_t j = w[1 + k];
            const int32_t cj = cur[j];
            if (cj == -1) {
                const unsigned long long pj = splitmix64(seed + (unsigned long long)j);
                if (!(pi > pj || (pi == pj && (uint32_t)i > j))) win = false;
            } else if (cj >= 0) {
                if (cj < 64) used |= 1ull << cj;
                else atomicOr(flags, 1u);
            }
        }
        if (win) {
            if (used == ~0ull) atomicOr(flags, 1u);  // would need a colour past 63
            next[i] = __ffsll((long long)~used) - 1;
        } else {
            cnt += 1ull;
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(left, cnt);
}

__global__ void colour_max_kernel(const int32_t *__restrict__ colour, int64_t n, int *cmax)
{
    int m = -1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        m = max(m, colour[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(cmax, m);
}

// Unchanged-tile skipping: for tile t (nodes 32t .. 32t+31), the tiles that
// hold its nodes and the neighbours of its free nodes, each with the mask of
// those nodes; (kHaloNever, 0) when more than kHaloEntries tiles are involved
// (such a tile is always computed).  One thread per tile.
__global__ void tile_halo_kernel(const uint32_t *__restrict__ node_off, const uint32_t *__restrict__ adj,
                                 int64_t n, int64_t ntiles, uint2 *halo)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    uint32_t ids[kHaloEntries], masks[kHaloEntries];
    int cnt = 1;
    ids[0] = (uint32_t)t;
    masks[0] = 0xffffffffu;
    bool over = false;
    for (int l = 0; l < 32 && !over; ++l) {
        const int64_t i = t * 32 + l;
        if (i >= n) break;
        const uint32_t off = node_off[i], meta = adj[off];
        if (meta & kMetaFixed) continue;
        const uint32_t deg = meta_degree(meta);
        for (uint32_t k = 0; k < deg; ++k) {
            const uint32_t j = adj[off + 1 + k];
            const uint32_t tj = j >> 5;
            int e = 0;
            while (e < cnt && ids[e] != tj) ++e;
            if (e == cnt) {
                if (cnt == kHaloEntries) {
                    over = true;
                    break;
                }
                ids[cnt] = tj;
                masks[cnt] = 0u;
                ++cnt;
            }
            masks[e] |= 1u << (j & 31);
        }
    }
    uint2 *h = halo + t * kHaloEntries;
    for (int e = 0; e < kHaloEntries; ++e)
        h[e] = over ? make_uint2(e == 0 ? kHaloNever : 0u, 0u)
                    : (e < cnt ? make_uint2(ids[e], masks[e]) : make_uint2(0u, 0u));
}

}  // namespace

sls_status build_tile_halo(sls_mesh *M, cudaStream_t s)
{
    if (!M->opt.skip_unchanged) return SLS_OK;
    const int64_t nt = (M->n + 31) / 32;
    GB_TRY(pool_alloc((void **)&M->halo, sizeof(uint2) * (size_t)kHaloEntries * (size_t)nt, s), "tile halo");
    for (int k = 0; k < 2; ++k) GB_TRY(pool_alloc((void **)&M->chg[k], sizeof(uint32_t) * (size_t)nt, s), "tile masks");
    GB_TRY(pool_alloc((void **)&M->accm, sizeof(uint32_t) * (size_t)nt, s), "tile masks");
    for (int k = 0; k < 2; ++k) GB_TRY(cudaMemsetAsync(M->chg[k], 0xff, sizeof(uint32_t) * (size_t)nt, s), "tile masks");
    GB_TRY(cudaMemsetAsync(M->accm, 0, sizeof(uint32_t) * (size_t)nt, s), "tile masks");
    tile_halo_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(M->node_off, M->adj, M->n, nt, M->halo);
    GB_TRY(cudaGetLastError(), "tile halo");
    GB_TRY(cudaStreamSynchronize(s), "tile halo");
    return SLS_OK;
}

namespace {

// One segment of the processing order: the free nodes of colour c (all free
// nodes when colour is null), in id order.
sls_status order_segment(sls_mesh *M, const int32_t *colour, int32_t c, uint32_t *dst, int64_t expect,
                         int64_t *count, cudaStream_t s)
{
    const int64_t n = M->n;
    const int64_t tiles = (n + kOrderTile - 1) / kOrderTile;
    DevBuf b_cnt, b_off;
    unsigned *cnt = nullptr;
    uint32_t *off = nullptr;
    sls_status st;
    if ((st = dalloc(b_cnt, (size_t)tiles, &cnt, "order counts", Alloc{false, s})) != SLS_OK) return st;
    if ((st = dalloc(b_off, (size_t)tiles + 1, &off, "order offsets", Alloc{false, s})) != SLS_OK) return st;
    order_count_kernel<<<(unsigned)tiles, kOrderTile, 0, s>>>(M->node_off, M->adj, n, colour, c, cnt);
    GB_TRY(cudaGetLastError(), "order count");
    unsigned long long total = 0ull;
    if ((st = scan_u32(cnt, tiles, off, &total, s)) != SLS_OK) return st;
    if (expect >= 0 && (int64_t)total > expect) return fail(SLS_ERR_INVALID, "processing order overflow");
    if (total > 0) {
        order_sort_kernel<<<(unsigned)tiles, kOrderTile, 0, s>>>(M->node_off, M->adj, n, colour, c, off, dst);
        GB_TRY(cudaGetLastError(), "order sort");
    }
    GB_TRY(cudaStreamSynchronize(s), "processing order");
    *count = (int64_t)total;
    return SLS_OK;
}

}  // namespace

namespace {

// ---- renumbering: Form B lists every colour class as a contiguous id range,
// Form A groups nodes by loop length inside windows of ids

__global__ void fixed_flag_kernel(const uint32_t *__restrict__ node_off, const uint32_t *__restrict__ adj, int64_t n,
                                  unsigned *flag)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        flag[i] = (__ldg(adj + __ldg(node_off + i)) & kMetaFixed) ? 1u : 0u;
}

// perm[base + scan[i]] = i for the flagged nodes, in id order.
__global__ void compact_kernel(const unsigned *__restrict__ flag, const uint32_t *__restrict__ scan, int64_t n,
                               int64_t base, uint32_t *perm)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        if (flag[i]) perm[base + scan[i]] = (uint32_t)i;
}

__global__ void inverse_kernel(const uint32_t *__restrict__ perm, int64_t n, uint32_t *inv)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) inv[perm[k]] = (uint32_t)k;
}

__global__ void record_len_kernel(const uint32_t *__restrict__ node_off, const uint32_t *__restrict__ perm, int64_t n,
                                  unsigned *len)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint32_t i = perm[k];
        len[k] = node_off[i + 1] - node_off[i];
    }
}

// The record of new node k is the record of old node perm[k] with its
// neighbour ids renumbered; the meta word and the triangle codes (positions
// in the neighbour list, whose order is kept) are copied as they are.
__global__ void remap_adj_kernel(const uint32_t *__restrict__ off_old, const uint32_t *__restrict__ adj_old,
                                 const uint32_t *__restrict__ perm, const uint32_t *__restrict__ inv,
                                 const uint32_t *__restrict__ off_new, int64_t n, uint32_t *__restrict__ adj_new)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const uint32_t *src = adj_old + off_old[perm[k]];
        uint32_t *dst = adj_new + off_new[k];
        const uint32_t meta = src[0];
        dst[0] = meta;
        if (meta & kMetaFixed) continue;
        const uint32_t deg = meta & 0xffffu, ntri = (meta >> 16) & 0x7fffu;
        for (uint32_t w = 1; w <= deg; ++w) dst[w] = inv[src[w]];
        for (uint32_t w = deg + 1; w <= deg + ntri; ++w) dst[w] = src[w];
    }
}

__global__ void remap_ids_kernel(int32_t *ids, int64_t count, const uint32_t *__restrict__ inv)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride)
        ids[t] = (int32_t)inv[ids[t]];
}

// Form B: inside every window of 128 positions of a colour class's id range
// (aligned to the class's start, as its ranged launches step through it) the
// class's nodes by (incident triangles, degree), ties by position: the same
// evening of a warp's loop lengths as Form A's grouped numbering, without
// mixing classes.  perm_in / perm_out: new position -> caller's id.
__global__ void __launch_bounds__(128) class_window_kernel(const uint32_t *__restrict__ perm_in,
                                                           const uint32_t *__restrict__ node_off,
                                                           const uint32_t *__restrict__ adj,
                                                           const int64_t *__restrict__ class_off,
                                                           const int64_t *__restrict__ win_off, int nclass,
                                                           uint32_t *__restrict__ perm_out)
{
    __shared__ uint32_t key[128];
    const int t = threadIdx.x;
    const int64_t nwin = win_off[nclass];
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        int c = 0;
        while (c + 1 < nclass && win_off[c + 1] <= w) ++c;
        const int64_t base = class_off[c] + 128 * (w - win_off[c]);
        const int64_t end = class_off[c + 1];
        const int len = end - base < 128 ? (int)(end - base) : 128;
        uint32_t k = 0xffffffffu, id = 0u;
        if (t < len) {
            id = perm_in[base + t];
            const uint32_t meta = __ldg(adj + __ldg(node_off + id));
            k = (meta_ntri(meta) << 16) | meta_degree(meta);
        }
        key[t] = k;
        __syncthreads();
        if (t < len) {
            int r = 0;
            for (int u = 0; u < len; ++u) {
                const uint32_t ku = key[u];
                r += (ku < k || (ku == k && u < t)) ? 1 : 0;
            }
            perm_out[base + r] = id;
        }
        __syncthreads();
    }
}

}  // namespace

// Renumbers the mesh by M->perm (new id -> caller's id, a permutation of
// [0, n) already on the device): fills M->inv and replaces the adjacency (the
// records in the new order, neighbour ids renumbered, each list's order
// kept, so every pass sums and tests exactly as before), the triangles and
// both coordinate arrays (which hold the creation coordinates).
static sls_status apply_renumbering(sls_mesh *M, cudaStream_t s)
{
    const int64_t n = M->n;
    const int grid = device_sm_count() * 8, block = 256;
    GB_TRY(pool_alloc((void **)&M->inv, sizeof(uint32_t) * (size_t)n, s), "renumbering");
    DevBuf b_len, b_off, b_adj;
    unsigned *len = nullptr;
    uint32_t *off_new = nullptr, *adj_new = nullptr;
    sls_status st;
    if ((st = dalloc(b_len, (size_t)n + 1, &len, "renumbering", Alloc{false, s})) != SLS_OK) return st;
    inverse_kernel<<<grid, block, 0, s>>>(M->perm, n, M->inv);
    record_len_kernel<<<grid, block, 0, s>>>(M->node_off, M->perm, n, len);
    GB_TRY(cudaGetLastError(), "renumbering");
    if ((st = dalloc(b_off, (size_t)n + 1, &off_new, "renumbering", Alloc{false, s})) != SLS_OK) return st;
    unsigned long long words = 0ull;
    if ((st = scan_u32(len, n, off_new, &words, s)) != SLS_OK) return st;
    if (words != M->adj_words) return fail(SLS_ERR_INVALID, "adjacency size mismatch in the renumbering");
    if ((st = dalloc(b_adj, (size_t)words, &adj_new, "renumbering", Alloc{false, s})) != SLS_OK) return st;
    remap_adj_kernel<<<grid, block, 0, s>>>(M->node_off, M->adj, M->perm, M->inv, off_new, n, adj_new);
    remap_ids_kernel<<<grid, block, 0, s>>>(M->tri, 3 * M->m, M->inv);
    GB_TRY(cudaGetLastError(), "renumbering");
    GB_TRY(launch_permute_coords(M->xy[0], M->xy[1], M->opt.layout, M->f32, n, M->perm, grid, s), "renumbering");
    GB_TRY(cudaMemcpyAsync(M->xy[0], M->xy[1], (M->f32 ? sizeof(float) : sizeof(double)) * 2 * (size_t)n,
                           cudaMemcpyDeviceToDevice, s), "renumbering");
    GB_TRY(cudaStreamSynchronize(s), "renumbering");
    pool_free(M->node_off, s);
    pool_free(M->adj, s);
    M->node_off = off_new;
    M->adj = adj_new;
    b_off.p = nullptr;  // now the mesh's
    b_adj.p = nullptr;
    return SLS_OK;
}

// A single mesh's grouped numbering (group_adjacency), with its triangles
// and both coordinate arrays (which hold the creation coordinates) moved to
// the new ids; fills M->perm and M->inv.
static sls_status group_by_degree(sls_mesh *M, cudaStream_t s)
{
    const int64_t n = M->n;
    const int grid = device_sm_count() * 8, block = 256;
    sls_status st = group_adjacency(n, &M->node_off, M->adj, false, s, &M->perm, &M->inv);
    if (st != SLS_OK) return st;
    remap_ids_kernel<<<grid, block, 0, s>>>(M->tri, 3 * M->m, M->inv);
    GB_TRY(cudaGetLastError(), "renumbering");
    GB_TRY(launch_permute_coords(M->xy[0], M->xy[1], M->opt.layout, M->f32, n, M->perm, grid, s), "renumbering");
    GB_TRY(cudaMemcpyAsync(M->xy[0], M->xy[1], (M->f32 ? sizeof(float) : sizeof(double)) * 2 * (size_t)n,
                           cudaMemcpyDeviceToDevice, s), "renumbering");
    GB_TRY(cudaStreamSynchronize(s), "renumbering");
    return SLS_OK;
}

// Form B: renumbers the mesh so that every colour class is a contiguous id
// range (the classes in order, each in its old id order, then the fixed
// nodes in id order): a sweep then reads and writes each class's nodes
// contiguously.  The colouring was computed on the caller's numbering, and
// the neighbour lists keep their order (only the ids change), so every pass
// computes what it computed before.  Fills M->perm (new -> caller's id) and
// M->inv; replaces the adjacency, the triangles and both coordinate arrays.
sls_status renumber_classes(sls_mesh *M, cudaStream_t s)
{
    const int64_t n = M->n;
    const int grid = device_sm_count() * 8, block = 256;
    GB_TRY(pool_alloc((void **)&M->perm, sizeof(uint32_t) * (size_t)n, s), "renumbering");
    // the free nodes by class: the processing order already lists them so
    if (M->n_free > 0)
        GB_TRY(cudaMemcpyAsync(M->perm, M->node_order, sizeof(uint32_t) * (size_t)M->n_free,
                               cudaMemcpyDeviceToDevice, s), "renumbering");
    DevBuf b_flag, b_scan;
    unsigned *flag = nullptr;
    uint32_t *scan = nullptr;
    sls_status st;
    if ((st = dalloc(b_flag, (size_t)n + 1, &flag, "renumbering", Alloc{false, s})) != SLS_OK) return st;
    if ((st = dalloc(b_scan, (size_t)n + 1, &scan, "renumbering", Alloc{false, s})) != SLS_OK) return st;
    fixed_flag_kernel<<<grid, block, 0, s>>>(M->node_off, M->adj, n, flag);
    GB_TRY(cudaGetLastError(), "renumbering");
    unsigned long long nfixed = 0ull;
    if ((st = scan_u32(flag, n, scan, &nfixed, s)) != SLS_OK) return st;
    if ((int64_t)nfixed + M->n_free != n) return fail(SLS_ERR_INVALID, "node count mismatch in the renumbering");
    compact_kernel<<<grid, block, 0, s>>>(flag, scan, n, M->n_free, M->perm);
    GB_TRY(cudaGetLastError(), "renumbering");
    const int nc = (int)M->colour_off.size() - 1;
    if (nc > 0 && M->n_free > 0 && groups_by_length(M->opt, n)) {
        // each class's windows grouped by loop length (see class_window_kernel)
        std::vector<int64_t> offs(2 * ((size_t)nc + 1));
        for (int c = 0; c <= nc; ++c) {
            offs[c] = M->colour_off[(size_t)c];
            offs[(size_t)nc + 1 + c] = c == 0 ? 0 : offs[(size_t)nc + c] + (offs[c] - offs[c - 1] + 127) / 128;
        }
        DevBuf b_perm2, b_offs;
        uint32_t *perm2 = nullptr;
        int64_t *d_offs = nullptr;
        if ((st = dalloc(b_perm2, (size_t)n, &perm2, "renumbering", Alloc{false, s})) != SLS_OK) return st;
        if ((st = dalloc(b_offs, offs.size(), &d_offs, "renumbering", Alloc{false, s})) != SLS_OK) return st;
        GB_TRY(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int64_t) * offs.size(), cudaMemcpyHostToDevice, s),
               "renumbering");
        GB_TRY(cudaMemcpyAsync(perm2, M->perm, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s),
               "renumbering");
        const int64_t nwin = offs[2 * (size_t)nc + 1];
        const int64_t cap = (int64_t)device_sm_count() * 16;
        class_window_kernel<<<(unsigned)(nwin < cap ? nwin : cap), 128, 0, s>>>(M->perm, M->node_off, M->adj, d_offs,
                                                                               d_offs + nc + 1, nc, perm2);
        GB_TRY(cudaGetLastError(), "renumbering");
        GB_TRY(cudaStreamSynchronize(s), "renumbering");  // offs is read from host memory
        b_perm2.p = M->perm;  // the plain class order goes back to the pool
        M->perm = perm2;
    }
    if ((st = apply_renumbering(M, s)) != SLS_OK) return st;
    pool_free(M->node_order, s);
    M->node_order = nullptr;
    return SLS_OK;
}

sls_status build_node_order(sls_mesh *M, cudaStream_t s)
{
    // Form A visits every node in index order: no list needed
    if (M->opt.form != 1) {
        return groups_nodes(M->opt, M->n) ? group_by_degree(M, s) : SLS_OK;
    }
    GB_TRY(pool_alloc((void **)&M->node_order, sizeof(uint32_t) * (size_t)(M->n_free > 0 ? M->n_free : 1), s),
           "processing order");
    // Form B: Jones-Plassmann colouring, then one order segment per colour
    const int64_t n = M->n;
    DevBuf b_col[2], b_cnt;
    int32_t *col[2] = {nullptr, nullptr};
    unsigned long long *cnt = nullptr;
    sls_status st;
    for (int k = 0; k < 2; ++k)
        if ((st = dalloc(b_col[k], (size_t)n, &col[k], "colours", Alloc{false, s})) != SLS_OK) return st;
    if ((st = dalloc(b_cnt, 2, &cnt, "colouring counters", Alloc{false, s})) != SLS_OK) return st;
    const int grid = device_sm_count() * 8, block = 256;
    colour_init_kernel<<<grid, block, 0, s>>>(M->node_off, M->adj, n, col[0]);
    GB_TRY(cudaGetLastError(), "colouring");
    int cur = 0;
    unsigned long long h[2] = {0ull, 0ull};
    for (int round = 0;; ++round) {
        if (round > 100000) return fail(SLS_ERR_INVALID, "colouring did not finish");
        GB_TRY(cudaMemcpyAsync(col[cur ^ 1], col[cur], sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s),
               "colouring");
        GB_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s), "colouring");
        colour_round_kernel<<<grid, block, 0, s>>>(M->node_off, M->adj, n, kColourSeed, col[cur], col[cur ^ 1], cnt,
                                                   reinterpret_cast<unsigned *>(cnt + 1));
        GB_TRY(cudaGetLastError(), "colouring round");
        GB_TRY(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, s), "colouring");
        GB_TRY(cudaStreamSynchronize(s), "colouring");
        cur ^= 1;
        if (h[1]) return fail(SLS_ERR_INVALID, "the coloured form needs more than 64 colours");
        if (h[0] == 0ull) break;
    }
    int *cmax = reinterpret_cast<int *>(cnt);
    GB_TRY(cudaMemsetAsync(cmax, 0xff, sizeof(int), s), "colouring");
    colour_max_kernel<<<grid, block, 0, s>>>(col[cur], n, cmax);
    int hmax = -1;
    GB_TRY(cudaMemcpyAsync(&hmax, cmax, sizeof hmax, cudaMemcpyDeviceToHost, s), "colouring");
    GB_TRY(cudaStreamSynchronize(s), "colouring");
    const int nc = hmax + 1;
    M->colour_off.assign((size_t)nc + 1, 0);
    int64_t at = 0;
    for (int c = 0; c < nc; ++c) {
        int64_t k = 0;
        if ((st = order_segment(M, col[cur], c, M->node_order + at, M->n_free - at, &k, s)) != SLS_OK) return st;
        at += k;
        M->colour_off[(size_t)c + 1] = at;
    }
    if (at != M->n_free) return fail(SLS_ERR_INVALID, "free-node count mismatch in the colouring");
    return renumber_classes(M, s);
}

// Builds the adjacency of a mesh whose coordinates (AoS) and triangles are
// already on the device.  On success out holds the node offsets and the
// adjacency words (allocated as `async` says; the caller owns them), the
// free-node count and D.  Returns SLS_ERR_NOT_FOUND (with nothing allocated)
// when a node has more incident triangles than the device build handles, so
// the caller can use the host build instead.  Synchronises only stream s.
sls_status build_device_adjacency(int64_t n, int64_t m, const double *d_xy, const int32_t *d_tri,
                                  const uint8_t *h_boundary, bool async, cudaStream_t s, DeviceAdjacency &out)
{
    out = DeviceAdjacency{};
    if (3 * m >= (int64_t(1) << 32)) return SLS_ERR_NOT_FOUND;
    const int sms = device_sm_count();
    const int grid = sms * 8, block = 256;
    const Alloc al{async, s};

    DevBuf b_flags, b_cnt, b_ptr, b_inc, b_nbtmp, b_words, b_fixed, b_deg, b_bnd, b_keys, b_off, b_adj;
    unsigned *flags = nullptr, *cnt = nullptr, *words = nullptr, *deg = nullptr;
    uint32_t *ptr = nullptr;
    int32_t *inc = nullptr, *nbtmp = nullptr;
    uint8_t *fixed = nullptr, *bnd = nullptr;
    unsigned long long *keys = nullptr;
    sls_status st;
    if ((st = dalloc(b_flags, 2, &flags, "build flags", al)) != SLS_OK) return st;
    if ((st = dalloc(b_keys, 8, &keys, "build keys", al)) != SLS_OK) return st;
    // keys: [0] first bad triangle, [1] first bad coordinate, [2..5] bbox, [6] free count
    GB_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(unsigned), s), "build");
    GB_TRY(cudaMemsetAsync(keys, 0xff, 2 * sizeof(unsigned long long), s), "build");
    validate_xy_kernel<<<grid, block, 0, s>>>(reinterpret_cast<const unsigned long long *>(d_xy), 2 * n, flags,
                                              keys + 1);
    validate_tri_kernel<<<grid, block, 0, s>>>(d_tri, m, n, flags, keys);
    GB_TRY(cudaGetLastError(), "validate");
    unsigned hflags = 0;
    unsigned long long hfirst[2] = {0, 0};
    GB_TRY(cudaMemcpyAsync(&hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s), "validate");
    GB_TRY(cudaMemcpyAsync(hfirst, keys, sizeof hfirst, cudaMemcpyDeviceToHost, s), "validate");
    GB_TRY(cudaStreamSynchronize(s), "validate");
    if (hflags & kErrFinite)
        return fail(SLS_ERR_INVALID, "coordinate " + std::to_string(hfirst[1]) + " is not finite");
    if (hflags & (kErrRange | kErrRepeat)) {
        const unsigned long long t = hfirst[0] >> 1;
        return fail(SLS_ERR_INVALID, "triangle " + std::to_string(t) +
                                         ((hfirst[0] & 1ull) ? " repeats a vertex" : " has a vertex id out of range"));
    }

    if ((st = dalloc(b_cnt, (size_t)n + 1, &cnt, "incidence counts", al)) != SLS_OK) return st;
    if ((st = dalloc(b_ptr, (size_t)n + 1, &ptr, "incidence offsets", al)) != SLS_OK) return st;
    if ((st = dalloc(b_inc, (size_t)(3 * m), &inc, "incidences", al)) != SLS_OK) return st;
    GB_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (n + 1), s), "build");
    count_kernel<<<grid, block, 0, s>>>(d_tri, 3 * m, cnt);
    GB_TRY(cudaGetLastError(), "count");
    unsigned long long total = 0ull;
    if ((st = scan_u32(cnt, n, ptr, &total, s, async)) != SLS_OK) return st;
    GB_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (n + 1), s), "build");
    scatter_kernel<<<grid, block, 0, s>>>(d_tri, 3 * m, ptr, cnt, inc);
    GB_TRY(cudaGetLastError(), "scatter");

    if ((st = dalloc(b_nbtmp, (size_t)(6 * m), &nbtmp, "neighbour scratch", al)) != SLS_OK) return st;
    if ((st = dalloc(b_words, (size_t)n + 1, &words, "word counts", al)) != SLS_OK) return st;
    if ((st = dalloc(b_fixed, (size_t)n, &fixed, "fixed flags", al)) != SLS_OK) return st;
    if ((st = dalloc(b_deg, (size_t)n, &deg, "degrees", al)) != SLS_OK) return st;
    if (h_boundary) {
        if ((st = dalloc(b_bnd, (size_t)n, &bnd, "boundary flags", al)) != SLS_OK) return st;
        GB_TRY(cudaMemcpyAsync(bnd, h_boundary, (size_t)n, cudaMemcpyHostToDevice, s), "upload flags");
    }
    node_pass1_kernel<<<grid, block, 0, s>>>(n, reinterpret_cast<const double2 *>(d_xy), d_tri, ptr, inc, bnd,
                                             nbtmp, words, fixed, deg, flags);
    GB_TRY(cudaGetLastError(), "node pass 1");
    GB_TRY(cudaMemcpyAsync(&hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s), "build");
    GB_TRY(cudaStreamSynchronize(s), "node pass 1");
    if (hflags & kErrManifold) return fail(SLS_ERR_NONMANIFOLD, "an edge is shared by more than two triangles");
    if (hflags & kErrTooMany) return SLS_ERR_NOT_FOUND;

    uint32_t *node_off = nullptr, *adj = nullptr;
    if ((st = dalloc(b_off, (size_t)n + 1, &node_off, "node offsets", al)) != SLS_OK) return st;
    unsigned long long wtotal = 0ull;
    if ((st = scan_u32(words, n, node_off, &wtotal, s, async)) != SLS_OK) return st;
    if (wtotal >= (1ull << 32)) return fail(SLS_ERR_INVALID, "adjacency exceeds 2^32 words");
    if ((st = dalloc(b_adj, (size_t)wtotal, &adj, "adjacency", al)) != SLS_OK) return st;
    node_pass2_kernel<<<grid, block, 0, s>>>(n, d_tri, ptr, inc, nbtmp, deg, fixed, node_off, adj);
    GB_TRY(cudaGetLastError(), "node pass 2");

    GB_TRY(cudaMemsetAsync(keys + 2, 0xff, 2 * sizeof(unsigned long long), s), "bbox");
    GB_TRY(cudaMemsetAsync(keys + 4, 0x00, 3 * sizeof(unsigned long long), s), "bbox");
    bbox_kernel<<<grid, block, 0, s>>>(reinterpret_cast<const double2 *>(d_xy), n, fixed, keys + 2, keys + 6);
    GB_TRY(cudaGetLastError(), "bbox");
    unsigned long long hk[5];
    GB_TRY(cudaMemcpyAsync(hk, keys + 2, sizeof hk, cudaMemcpyDeviceToHost, s), "bbox");
    GB_TRY(cudaStreamSynchronize(s), "build");
    auto unkey = [](unsigned long long k) {
        const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
        double v;
        std::memcpy(&v, &b, sizeof v);
        return v;
    };
    const double xmin = unkey(hk[0]), ymin = unkey(hk[1]), xmax = unkey(hk[2]), ymax = unkey(hk[3]);
    out.diag = bbox_diagonal(xmin, xmax, ymin, ymax);
    out.n_free = (int64_t)hk[4];
    out.adj_words = wtotal;
    out.node_off = node_off;
    out.adj = adj;
    b_off.p = nullptr;  // handed to the caller
    b_adj.p = nullptr;
    return SLS_OK;
}

sls_status build_device_mesh(sls_mesh *M, const double *d_xy, const int32_t *d_tri, const uint8_t *h_boundary,
                             cudaStream_t s)
{
    DeviceAdjacency da;
    sls_status st = build_device_adjacency(M->n, M->m, d_xy, d_tri, h_boundary, false, s, da);
    if (st != SLS_OK) return st;
    M->node_off = da.node_off;
    M->adj = da.adj;
    M->adj_words = da.adj_words;
    M->n_free = da.n_free;
    M->diag = da.diag;
    return SLS_OK;
}

}  // namespace sls
