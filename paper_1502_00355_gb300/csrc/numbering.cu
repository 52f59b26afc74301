// numbering.cu -- Form A's grouped internal numbering of a mesh.
//
// The lanes of a warp run in step, so the screened pass's neighbour loop
// runs to the largest degree among a warp's 32 nodes and its triangle loop to
// the largest triangle count.  Listing the nodes of every window of 128
// consecutive ids (the ids one block of 128 threads covers in one step of its
// grid stride) by incident-triangle count and degree evens those counts
// within a warp while the window, and so the block's gathers, stay where
// they are.  The pass then computes the same bits: only ids change, every
// neighbour list keeps its order and hence the summation order of Eq. 2.
#include <string>

#include "api_common.h"
#include "device.cuh"

namespace sls {
namespace {

constexpr int kGroupWindow = 128;  // the ids one block of the pass covers per grid-stride step

// Inside each window of kGroupWindow consecutive ids, the window's nodes by
// (incident triangles, degree), fixed nodes last, ties by id (a stable
// counting rank over the window's keys in shared memory): perm[new] = old,
// inv[old] = new and off_new[new] = off_old[old], off_new[n] = off_old[n].
__global__ void __launch_bounds__(kGroupWindow) window_group_kernel(const uint32_t *__restrict__ node_off,
                                                                    const uint32_t *__restrict__ adj, int64_t n,
                                                                    uint32_t *__restrict__ perm,
                                                                    uint32_t *__restrict__ inv,
                                                                    uint32_t *__restrict__ off_new)
{
    __shared__ uint32_t key[kGroupWindow];
    const int t = threadIdx.x;
    const int64_t nwin = (n + kGroupWindow - 1) / kGroupWindow;
    if (blockIdx.x == 0 && t == 0) off_new[n] = node_off[n];
    for (int64_t w = blockIdx.x; w < nwin; w += gridDim.x) {
        const int64_t base = w * kGroupWindow;
        const int len = n - base < kGroupWindow ? (int)(n - base) : kGroupWindow;
        uint32_t k = 0xffffffffu, off = 0u;
        if (t < len) {
            off = __ldg(node_off + base + t);
            const uint32_t meta = __ldg(adj + off);
            k = (meta & kMetaFixed) ? 0xfffffffeu : (meta_ntri(meta) << 16) | meta_degree(meta);
        }
        key[t] = k;
        __syncthreads();
        if (t < len) {
            int r = 0;
            for (int u = 0; u < len; ++u) {
                const uint32_t ku = key[u];
                r += (ku < k || (ku == k && u < t)) ? 1 : 0;
            }
            perm[base + r] = (uint32_t)(base + t);
            inv[base + t] = (uint32_t)(base + r);
            off_new[base + r] = off;
        }
        __syncthreads();
    }
}

// Neighbour ids of every record renumbered where the record lies (Form A
// keeps its records in place; the list order, hence the summation order, is
// unchanged).
__global__ void remap_in_place_kernel(const uint32_t *__restrict__ node_off, uint32_t *__restrict__ adj, int64_t n,
                                      const uint32_t *__restrict__ inv)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t *rec = adj + node_off[i];
        const uint32_t meta = rec[0];
        if (meta & kMetaFixed) continue;
        const uint32_t deg = meta_degree(meta);
        for (uint32_t w = 1; w <= deg; ++w) rec[w] = inv[rec[w]];
    }
}


}  // namespace

// Form A's grouped numbering of a built adjacency (n nodes; *node_off and
// adj on the device): inside every window of kGroupWindow consecutive ids
// the nodes are listed by incident-triangle count and degree.  The pass's
// neighbour loop runs to the largest degree in a warp and its triangle loop
// to the largest count (the lanes run in step), so 32 nodes of similar
// counts spend fewer idle trips; the windows are the id ranges a block covers
// together, so their gathers share the block's L1 as before.  The records
// stay where they are (a window's records are contiguous either way): their
// neighbour ids are renumbered in place and *node_off is replaced by the
// permuted offsets (the old array returned to the pool).  *perm_out (new id
// -> old id) and, when inv_out is not NULL, *inv_out (old -> new) come from
// the library's pool on s and belong to the caller; coordinates and
// triangles are the caller's to move.  Synchronises s unless `async`.
sls_status group_adjacency(int64_t n, uint32_t **node_off, uint32_t *adj, bool async, cudaStream_t s,
                           uint32_t **perm_out, uint32_t **inv_out)
{
    uint32_t *perm = nullptr, *inv = nullptr, *off_new = nullptr;
    auto give_back = [&](cudaError_t e, const char *what) {
        pool_free(perm, s);
        pool_free(inv, s);
        pool_free(off_new, s);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(SLS_ERR_OOM, std::string("device allocation failed: ") + what);
        }
        return cuda_fail(e, what);
    };
    cudaError_t e = pool_alloc((void **)&perm, sizeof(uint32_t) * (size_t)n, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&inv, sizeof(uint32_t) * (size_t)n, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&off_new, sizeof(uint32_t) * (size_t)(n + 1), s);
    if (e != cudaSuccess) return give_back(e, "renumbering");
    const int grid = device_sm_count() * 8, block = 256;
    const int64_t nwin = (n + kGroupWindow - 1) / kGroupWindow;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    window_group_kernel<<<(unsigned)(nwin < cap ? nwin : cap), kGroupWindow, 0, s>>>(*node_off, adj, n, perm,
                                                                                    inv, off_new);
    remap_in_place_kernel<<<grid, block, 0, s>>>(*node_off, adj, n, inv);
    e = cudaGetLastError();
    if (e == cudaSuccess && !async) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return give_back(e, "renumbering");
    pool_free(*node_off, s);
    *node_off = off_new;
    *perm_out = perm;
    if (inv_out) *inv_out = inv;
    else pool_free(inv, s);
    return SLS_OK;
}

}  // namespace sls
