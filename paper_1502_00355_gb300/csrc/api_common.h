// api_common.h -- the mesh handle and the helpers behind the C ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

struct sls_mesh {
    sls_options opt{};
    int64_t n = 0, m = 0, n_free = 0;
    double diag = 0.0;            // bounding-box diagonal of the creation coordinates
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    double *xy[2] = {nullptr, nullptr};  // the two coordinate arrays (2n doubles each, 2n floats when f32)
    bool f32 = false;             // binary32 coordinates and arithmetic
    int cur = 0;                  // which of the two holds the current coordinates
    uint32_t *node_off = nullptr; // n+1
    uint32_t *adj = nullptr;      // node_off[n] words
    uint64_t adj_words = 0;
    uint32_t *node_order = nullptr;  // n_free: processing order of the free nodes (Form A: none)
    uint32_t *perm = nullptr;     // renumbered mesh: internal id -> the caller's id (Form B: colour
                                  // classes contiguous; Form A: grouped by loop length in windows)
    uint32_t *inv = nullptr;      // the caller's id -> internal id
    std::vector<int64_t> colour_off; // segments of node_order: one per colour (Form B), else one
    int32_t *tri = nullptr;       // 3m, for the histogram
    sls::PassStats *stats = nullptr;  // one record per pass of a call
    int stats_cap = 0;
    sls::PassStats *h_stats = nullptr;  // pinned, one record
    uint8_t *accept = nullptr;    // n, when record_accept
    uint2 *halo = nullptr;        // skip_unchanged: kHaloEntries (tile, mask) pairs per 32-node tile
    uint32_t *chg[2] = {nullptr, nullptr};  // per tile: nodes changed by the last two passes
    uint32_t *accm = nullptr;     // per tile: nodes accepted when the tile was last computed
    size_t l2_persist = 0;        // l2_window: persisting L2 bytes set aside for this context
    size_t l2_win_max = 0;        //            largest access-policy window the device accepts
    unsigned *xfer_bad = nullptr; // gather/scatter: set when an id was out of range
    int block = 256, grid = 0;
    bool screened = true;         // screened kernel (else the plain FP64 kernel)
    sls_info last{};
};

namespace sls {

sls_status cuda_fail(cudaError_t e, const char *what);
int device_sm_count();
// Unique id of the calling thread's current CUDA context, 0 when there is
// none.  Per-device set-up (constant memory, symbol addresses) is keyed on it,
// so a context created after cudaDeviceReset is set up again.
unsigned long long current_context_id();
// Loads the allocation-free entry point's scratch array on the current
// device (noalloc.cu); sls_mesh_create calls it, so sls_smooth_noalloc on a
// mesh never loads code or data itself.
sls_status noalloc_prepare();
sls_options resolve_options(const sls_options *opt);
sls_status check_options(const sls_options &o);

sls_status mesh_upload(sls_mesh *M, const HostMesh &hm, const double *xy, const int32_t *tri,
                       const sls_options &o);
// Uploads coordinates and triangles and builds the adjacency on the device
// (host build as a fallback for very high-valence nodes).
sls_status mesh_create_on_device(sls_mesh *M, const double *xy, int64_t n, const int32_t *tri, int64_t m,
                                 const uint8_t *boundary, const sls_options &o);
// Adjacency built on the device (mesh_build_gpu.cu).
struct DeviceAdjacency {
    uint32_t *node_off = nullptr;  // n+1
    uint32_t *adj = nullptr;       // adj_words
    uint64_t adj_words = 0;
    int64_t n_free = 0;
    double diag = 0.0;
};
// Validates the mesh and builds its adjacency from device copies of the
// coordinates (AoS) and triangles; every allocation is stream-ordered on s
// when `async` (the caller then frees the outputs with cudaFreeAsync).
// SLS_ERR_NOT_FOUND = a node is in too many triangles: use the host build.
sls_status build_device_adjacency(int64_t n, int64_t m, const double *d_xy, const int32_t *d_tri,
                                  const uint8_t *h_boundary, bool async, cudaStream_t s, DeviceAdjacency &out);
// Device memory of the handles (memory.cu): stream-ordered allocations from
// the library's pool on the current device, which keeps freed memory for
// later handles (sls_trim_memory returns it).  Allocate and free on the
// stream that uses the buffer; pool_free ignores NULL.
cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
// Form A's grouped numbering of a built adjacency (mesh_build_gpu.cu): nodes
// listed by incident-triangle count and degree inside windows of 128 ids;
// neighbour ids renumbered in place, *node_off replaced by the permuted
// offsets; *perm_out (new -> old id) and, if inv_out is not NULL, *inv_out
// (old -> new) allocated as `async` says, the caller's to free.
sls_status group_adjacency(int64_t n, uint32_t **node_off, uint32_t *adj, bool async, cudaStream_t s,
                           uint32_t **perm_out, uint32_t **inv_out);
// Whether options o group the nodes of a mesh of n nodes by loop length
// (FP64 only: the binary32 pass's loops are per lane, and there the grouping
// only costs locality).
inline bool groups_by_length(const sls_options &o, int64_t n)
{
    return o.precision != 32 && !o.skip_unchanged && (o.numbering == 2 || (o.numbering == 0 && n >= (int64_t(1) << 20)));
}
// Whether options o renumber a Form-A mesh of n nodes (grouped numbering).
inline bool groups_nodes(const sls_options &o, int64_t n) { return o.form == 0 && groups_by_length(o, n); }
// Device adjacency build of a mesh handle; SLS_ERR_NOT_FOUND = use the host build.
sls_status build_device_mesh(sls_mesh *M, const double *d_xy, const int32_t *d_tri, const uint8_t *h_boundary,
                             cudaStream_t s);
// The processing order of the free nodes, from the adjacency on the device
// (mesh_build_gpu.cu): fills M->node_order.
sls_status build_node_order(sls_mesh *M, cudaStream_t s);
// The tile lists and masks of unchanged-tile skipping (mesh_build_gpu.cu),
// when opt.skip_unchanged is set.
sls_status build_tile_halo(sls_mesh *M, cudaStream_t s);
void mesh_release(sls_mesh *M);
sls_status mesh_run(sls_mesh *M, int32_t max_iter, double tol_rel, sls_info &info);
sls_status mesh_download(const sls_mesh *M, double *xy_out, bool dst_is_device);
sls_status mesh_set_coords(sls_mesh *M, const double *xy, bool src_is_device);
// Device gather (scatter = false: buf <- current coordinates of the listed
// nodes) or scatter (buf -> both coordinate arrays) of k nodes; returns when done.
sls_status mesh_transfer_nodes(sls_mesh *M, const int32_t *idx, int64_t k, double *buf, bool scatter);
sls_status mesh_histogram(const sls_mesh *M, int nbins, double lo, double hi, int64_t *counts,
                          double *qmin, double *qmean);

// (tol * D)^2 with the tolerance stop's exact rounding.
inline double tolerance_threshold(double tol_rel, double diag)
{
    double a = tol_rel * diag;
    return a * a;
}

}  // namespace sls
