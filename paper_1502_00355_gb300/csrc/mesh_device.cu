// mesh_device.cu -- device memory, pass scheduling and transfers of a mesh handle.
#include <algorithm>
#include <cstring>
#include <vector>

#include "api_common.h"
#include "kernels.h"

namespace sls {

#define SLS_CUDA_TRY(expr, what)                 \
    do {                                         \
        cudaError_t e_ = (expr);                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// A buffer of mesh M from the library's pool, on the mesh's stream.
static sls_status dev_alloc(const sls_mesh *M, void **p, size_t bytes, const char *what)
{
    cudaError_t e = pool_alloc(p, bytes, M->stream);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(SLS_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    if (e != cudaSuccess) return cuda_fail(e, what);
    return SLS_OK;
}

// Host interleaved -> SoA (x[n] then y[n]).
static void to_soa(const double *xy, int64_t n, std::vector<double> &tmp)
{
    tmp.resize(2 * n);
    for (int64_t i = 0; i < n; ++i) {
        tmp[i] = xy[2 * i];
        tmp[n + i] = xy[2 * i + 1];
    }
}

// Common set-up of a handle: stream, statistics, accept mask, launch shape.
static sls_status mesh_setup(sls_mesh *M, const sls_options &o)
{
    M->opt = o;
    SLS_CUDA_TRY(cudaGetDevice(&M->device), "cudaGetDevice");
    if (o.stream) {
        M->stream = (cudaStream_t)o.stream;
    } else {
        SLS_CUDA_TRY(cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        M->own_stream = true;
    }
    sls_status st;
    M->stats_cap = 256;
    if ((st = dev_alloc(M, (void **)&M->stats, sizeof(PassStats) * M->stats_cap, "pass statistics")) != SLS_OK) return st;
    SLS_CUDA_TRY(cudaMallocHost((void **)&M->h_stats, sizeof(PassStats)), "cudaMallocHost");
    if (o.record_accept) {
        if ((st = dev_alloc(M, (void **)&M->accept, (size_t)M->n, "accept mask")) != SLS_OK) return st;
        SLS_CUDA_TRY(cudaMemsetAsync(M->accept, 0, (size_t)M->n, M->stream), "cudaMemset");
    }
    M->cur = 0;
    M->f32 = o.precision == 32;
    M->block = o.block_size;
    M->screened = o.kernel != SLS_KERNEL_FP64 && !M->f32;
    if (M->screened && M->block > 128) M->block = 128;  // the screened kernel is built for <= 128
    if (M->f32 && M->block > 256) M->block = 256;  // the binary32 kernel is built for <= 256
    if (o.l2_window) {
        // Persisting L2 for the coordinates each pass gathers from: the
        // context's persisting carve-out covers at most one coordinate array.
        int maxp = 0, maxw = 0;
        cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, M->device);
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, M->device);
        const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
        M->l2_persist = std::min((size_t)(maxp > 0 ? maxp : 0), cbytes);
        M->l2_win_max = (size_t)(maxw > 0 ? maxw : 0);
        if (M->l2_persist > 0 && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, M->l2_persist) != cudaSuccess) {
            cudaGetLastError();
            M->l2_persist = 0;
        }
    }
    sls_status pst = noalloc_prepare();
    if (pst != SLS_OK) return pst;
    M->grid = device_sm_count() * (M->f32        ? pass_f32_occupancy(o.layout, M->block)
                                   : M->screened ? pass_screened_occupancy(o.layout, M->block)
                                                 : pass_fp64_occupancy(o.layout, M->block));
    return SLS_OK;
}

// Binary32 meshes: the coordinates, built as doubles in the mesh's layout,
// are rounded to floats; the two arrays then hold 2n floats each.
static sls_status narrow_coordinates(sls_mesh *M)
{
    if (!M->f32) return SLS_OK;
    const size_t fbytes = sizeof(float) * 2 * (size_t)M->n;
    float *f[2] = {nullptr, nullptr};
    sls_status st;
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(M, (void **)&f[b], fbytes, "coordinates")) != SLS_OK) {
            pool_free(f[0], M->stream);
            return st;
        }
    const int grid = device_sm_count() * 4;
    const double *aos = M->xy[0];
    if (M->opt.layout == 1) {  // interleave first (xy[1] holds a copy of xy[0])
        SLS_CUDA_TRY(launch_soa_to_aos(M->xy[0], M->xy[1], M->n, grid, M->stream), "interleave");
        aos = M->xy[1];
    }
    SLS_CUDA_TRY(launch_narrow(aos, f[0], M->n, M->opt.layout, grid, M->stream), "narrow");
    SLS_CUDA_TRY(cudaMemcpyAsync(f[1], f[0], fbytes, cudaMemcpyDeviceToDevice, M->stream), "copy coordinates");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "narrow");
    for (int b = 0; b < 2; ++b) {
        pool_free(M->xy[b], M->stream);
        M->xy[b] = reinterpret_cast<double *>(f[b]);
    }
    return SLS_OK;
}

sls_status mesh_upload(sls_mesh *M, const HostMesh &hm, const double *xy, const int32_t *tri,
                       const sls_options &o)
{
    M->n = hm.n;
    M->m = hm.m;
    M->n_free = hm.n_free;
    M->diag = hm.diag;
    M->adj_words = hm.node_off[hm.n];
    sls_status st = mesh_setup(M, o);
    if (st != SLS_OK) return st;
    const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(M, (void **)&M->xy[b], cbytes, "coordinates")) != SLS_OK) return st;
    if ((st = dev_alloc(M, (void **)&M->node_off, sizeof(uint32_t) * (M->n + 1), "node offsets")) != SLS_OK) return st;
    if ((st = dev_alloc(M, (void **)&M->adj, sizeof(uint32_t) * M->adj_words, "adjacency")) != SLS_OK) return st;
    if ((st = dev_alloc(M, (void **)&M->tri, sizeof(int32_t) * 3 * (size_t)M->m, "triangles")) != SLS_OK) return st;
    if (o.layout == 0) {
        SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[0], xy, cbytes, cudaMemcpyHostToDevice, M->stream), "upload coordinates");
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "upload coordinates");
    } else {
        std::vector<double> tmp;
        to_soa(xy, M->n, tmp);
        SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[0], tmp.data(), cbytes, cudaMemcpyHostToDevice, M->stream), "upload coordinates");
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "upload coordinates");
    }
    SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[1], M->xy[0], cbytes, cudaMemcpyDeviceToDevice, M->stream), "copy coordinates");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->node_off, hm.node_off.data(), sizeof(uint32_t) * (M->n + 1),
                                 cudaMemcpyHostToDevice, M->stream), "upload offsets");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->adj, hm.adj.data(), sizeof(uint32_t) * M->adj_words,
                                 cudaMemcpyHostToDevice, M->stream), "upload adjacency");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->tri, tri, sizeof(int32_t) * 3 * (size_t)M->m,
                                 cudaMemcpyHostToDevice, M->stream), "upload triangles");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "upload");
    if ((st = narrow_coordinates(M)) != SLS_OK) return st;
    if ((st = build_node_order(M, M->stream)) != SLS_OK) return st;
    return build_tile_halo(M, M->stream);
}

sls_status mesh_create_on_device(sls_mesh *M, const double *xy, int64_t n, const int32_t *tri, int64_t m,
                                 const uint8_t *boundary, const sls_options &o)
{
    M->n = n;
    M->m = m;
    sls_status st = mesh_setup(M, o);
    if (st != SLS_OK) return st;
    const size_t cbytes = sizeof(double) * 2 * (size_t)n;
    for (int b = 0; b < 2; ++b)
        if ((st = dev_alloc(M, (void **)&M->xy[b], cbytes, "coordinates")) != SLS_OK) return st;
    if ((st = dev_alloc(M, (void **)&M->tri, sizeof(int32_t) * 3 * (size_t)m, "triangles")) != SLS_OK) return st;
    // interleaved coordinates go to xy[0] (AoS) or xy[1] (staging for SoA)
    double *aos = o.layout == 0 ? M->xy[0] : M->xy[1];
    SLS_CUDA_TRY(cudaMemcpyAsync(aos, xy, cbytes, cudaMemcpyHostToDevice, M->stream), "upload coordinates");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->tri, tri, sizeof(int32_t) * 3 * (size_t)m, cudaMemcpyHostToDevice, M->stream),
                 "upload triangles");
    st = build_device_mesh(M, aos, M->tri, boundary, M->stream);
    if (st == SLS_ERR_NOT_FOUND) {
        // a node with more incident triangles than the device build handles
        HostMesh hm;
        st = build_host_mesh(xy, n, tri, m, boundary, hm);
        if (st != SLS_OK) return st;
        pool_free(M->node_off, M->stream);
        pool_free(M->adj, M->stream);
        M->node_off = nullptr;
        M->adj = nullptr;
        M->n_free = hm.n_free;
        M->diag = hm.diag;
        M->adj_words = hm.node_off[hm.n];
        if ((st = dev_alloc(M, (void **)&M->node_off, sizeof(uint32_t) * (n + 1), "node offsets")) != SLS_OK) return st;
        if ((st = dev_alloc(M, (void **)&M->adj, sizeof(uint32_t) * M->adj_words, "adjacency")) != SLS_OK) return st;
        SLS_CUDA_TRY(cudaMemcpyAsync(M->node_off, hm.node_off.data(), sizeof(uint32_t) * (n + 1),
                                     cudaMemcpyHostToDevice, M->stream), "upload offsets");
        SLS_CUDA_TRY(cudaMemcpyAsync(M->adj, hm.adj.data(), sizeof(uint32_t) * M->adj_words,
                                     cudaMemcpyHostToDevice, M->stream), "upload adjacency");
    } else if (st != SLS_OK) {
        return st;
    }
    if (o.layout == 1)
        SLS_CUDA_TRY(launch_aos_to_soa(M->xy[1], M->xy[0], n, device_sm_count() * 4, M->stream), "split");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[1], M->xy[0], cbytes, cudaMemcpyDeviceToDevice, M->stream), "copy coordinates");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "mesh create");
    if ((st = narrow_coordinates(M)) != SLS_OK) return st;
    if ((st = build_node_order(M, M->stream)) != SLS_OK) return st;
    return build_tile_halo(M, M->stream);
}

void mesh_release(sls_mesh *M)
{
    if (M->stream) cudaStreamSynchronize(M->stream);
    pool_free(M->xy[0], M->stream);
    pool_free(M->xy[1], M->stream);
    pool_free(M->node_off, M->stream);
    pool_free(M->adj, M->stream);
    pool_free(M->node_order, M->stream);
    pool_free(M->perm, M->stream);
    pool_free(M->inv, M->stream);
    pool_free(M->tri, M->stream);
    pool_free(M->stats, M->stream);
    pool_free(M->accept, M->stream);
    pool_free(M->halo, M->stream);
    pool_free(M->chg[0], M->stream);
    pool_free(M->chg[1], M->stream);
    pool_free(M->accm, M->stream);
    pool_free(M->xfer_bad, M->stream);
    if (M->h_stats) cudaFreeHost(M->h_stats);
    if (M->own_stream && M->stream) cudaStreamDestroy(M->stream);
    M->stream = nullptr;
}

// Access-policy window of the handle's stream: `bytes` from `base` persist in
// L2 (the share that fits the carve-out), the rest streams; bytes = 0 clears
// it.  Best effort: a refusal leaves the ordinary caching.
static void set_l2_window(const sls_mesh *M, const void *base, size_t bytes)
{
    if (M->l2_persist == 0 || M->l2_win_max == 0) return;
    cudaStreamAttrValue v{};
    bytes = std::min(bytes, M->l2_win_max);
    v.accessPolicyWindow.base_ptr = bytes ? const_cast<void *>(base) : nullptr;
    v.accessPolicyWindow.num_bytes = bytes;
    v.accessPolicyWindow.hitRatio = bytes ? (float)std::min(1.0, (double)M->l2_persist / (double)bytes) : 0.0f;
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    if (cudaStreamSetAttribute(M->stream, cudaStreamAttributeAccessPolicyWindow, &v) != cudaSuccess) cudaGetLastError();
}

static cudaError_t launch_pass(const sls_mesh *M, const PassArgs &a)
{
    if (M->opt.l2_window) set_l2_window(M, a.in, (M->f32 ? sizeof(float) : sizeof(double)) * 2 * (size_t)M->n);
    if (M->f32) return launch_pass_f32(a, M->opt.layout, M->block, M->grid, M->stream);
    return M->screened ? launch_pass_screened(a, M->opt.layout, M->block, M->grid, M->stream)
                       : launch_pass_fp64(a, M->opt.layout, M->block, M->grid, M->stream);
}

sls_status mesh_run(sls_mesh *M, int32_t max_iter, double tol_rel, sls_info &info)
{
    info = sls_info{};
    if (max_iter == 0) return SLS_OK;
    if (M->stats_cap < max_iter) {
        cudaStreamSynchronize(M->stream);
        pool_free(M->stats, M->stream);
        M->stats = nullptr;
        int cap = std::max(max_iter, 2 * M->stats_cap);
        sls_status st = dev_alloc(M, (void **)&M->stats, sizeof(PassStats) * cap, "pass statistics");
        if (st != SLS_OK) {
            M->stats_cap = 0;
            return st;
        }
        M->stats_cap = cap;
    }
    SLS_CUDA_TRY(cudaMemsetAsync(M->stats, 0, sizeof(PassStats) * max_iter, M->stream), "cudaMemset");
    const bool tol_active = tol_rel > 0.0;
    const double thr = tolerance_threshold(tol_rel, M->diag);
    unsigned long long thr_bits;
    std::memcpy(&thr_bits, &thr, sizeof thr_bits);

    PassArgs a{};
    a.node_off = M->node_off;
    a.adj = M->adj;
    a.n = M->n;
    a.order = M->node_order;
    a.norder = M->n_free;
    a.stats = M->stats;
    a.strict = M->opt.accept_strict;
    a.tol_active = tol_active ? 1 : 0;
    a.thr_bits = thr_bits;
    a.accept = M->accept;
    const bool form_b = M->opt.form == 1;
    const int cb = form_b ? 0 : M->opt.copy_back;
    const int chunk = M->opt.passes_per_check;
    const int nseg = (int)M->colour_off.size() - 1;
    int launched = 0;
    int64_t kernels = 0;
    while (launched < max_iter) {
        const int end = std::min(launched + chunk, (int)max_iter);
        for (int q = launched; q < end; ++q) {
            a.q = q;
            if (form_b) {
                // Form B: the colour classes in turn, in place (Eq. 3).  A
                // mesh without free nodes has no class; one launch over an
                // empty list still records the sweep, as Form A does.
                // the mesh is renumbered: class c is the id range colour_off[c] ..
                a.in = a.out = M->xy[M->cur];
                for (int c = 0; c < std::max(nseg, 1); ++c) {
                    a.order = nullptr;
                    a.ranged = 1;
                    a.first = nseg > 0 ? M->colour_off[c] : 0;
                    a.count = nseg > 0 ? M->colour_off[c + 1] - M->colour_off[c] : 0;
                    SLS_CUDA_TRY(launch_pass(M, a), "pass kernel");
                    ++kernels;
                }
                continue;
            }
            const int src = cb ? M->cur : (M->cur ^ (q & 1));
            a.in = M->xy[src];
            a.out = M->xy[src ^ 1];
            a.order = nullptr;
            a.norder = 0;
            if (M->halo) {  // unchanged-tile skipping from the second pass of a call on
                a.halo = M->halo;
                a.chg_prev = M->chg[(q + 1) & 1];
                a.chg_cur = M->chg[q & 1];
                a.accm = M->accm;
                a.skip = q > 0 ? 1 : 0;
            }
            SLS_CUDA_TRY(launch_pass(M, a), "pass kernel");
            ++kernels;
            if (cb) {
                SLS_CUDA_TRY(M->f32 ? launch_copy_back_f32(reinterpret_cast<const float *>(M->xy[src ^ 1]),
                                                           reinterpret_cast<float *>(M->xy[src]), 2 * M->n,
                                                           M->stats, q, device_sm_count() * 4, M->stream)
                                    : launch_copy_back(M->xy[src ^ 1], M->xy[src], 2 * M->n, M->stats, q,
                                                       device_sm_count() * 4, M->stream),
                             "copy-back kernel");
                ++kernels;
            }
        }
        launched = end;
        if (tol_active && launched < max_iter) {
            SLS_CUDA_TRY(cudaMemcpyAsync(M->h_stats, M->stats + launched - 1, sizeof(PassStats),
                                         cudaMemcpyDeviceToHost, M->stream), "read pass statistics");
            SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "pass");
            if (M->h_stats->executed == 0u || M->h_stats->maxd2_bits < thr_bits) break;
        }
    }
    if (M->opt.l2_window && M->l2_persist) {  // leave no persisting lines behind
        set_l2_window(M, nullptr, 0);
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "pass");
        if (cudaCtxResetPersistingL2Cache() != cudaSuccess) cudaGetLastError();
    }
    std::vector<PassStats> hs(launched);
    SLS_CUDA_TRY(cudaMemcpyAsync(hs.data(), M->stats, sizeof(PassStats) * launched,
                                 cudaMemcpyDeviceToHost, M->stream), "read pass statistics");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "passes");
    int it = 0;
    long long fb = 0, sk = 0;
    for (; it < launched && hs[it].executed; ++it) {
        fb += (long long)hs[it].fallbacks;
        sk += (long long)hs[it].nodes_skipped;
    }
    info.iterations = it;
    info.fp64_fallbacks = fb;
    info.nodes_skipped = sk;
    info.launches = kernels;
    if (it > 0) {
        const PassStats &l = hs[it - 1];
        info.accepted_last = (int64_t)l.nacc;
        std::memcpy(&info.max_d2_last, &l.maxd2_bits, sizeof(double));
        info.converged = (tol_active && l.maxd2_bits < thr_bits) ? 1 : 0;
    }
    if (!cb && !form_b) M->cur ^= (it & 1);
    return SLS_OK;
}

sls_status mesh_download(const sls_mesh *M, double *xy_out, bool dst_is_device)
{
    const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
    const double *src = M->xy[M->cur];
    if (M->perm) {
        // renumbered mesh: back to the caller's numbering (and to interleaved
        // doubles) on the device.  For a host destination an FP64 mesh stages
        // it in its other coordinate array (nothing reads that array before a
        // pass rewrites its free nodes) and then copies the current one back
        // over it, so that its fixed nodes hold their values again
        const bool stage = !dst_is_device && !M->f32;
        double *d = dst_is_device ? xy_out : (stage ? M->xy[M->cur ^ 1] : nullptr);
        sls_status st;
        if (!d && (st = dev_alloc(M, (void **)&d, cbytes, "download")) != SLS_OK) return st;
        cudaError_t e = launch_unpermute_to_aos(src, M->opt.layout, M->f32, M->n, M->perm, d,
                                                device_sm_count() * 4, M->stream);
        if (e == cudaSuccess && !dst_is_device)
            e = cudaMemcpyAsync(xy_out, d, cbytes, cudaMemcpyDeviceToHost, M->stream);
        if (e == cudaSuccess && stage) e = cudaMemcpyAsync(d, src, cbytes, cudaMemcpyDeviceToDevice, M->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
        if (!dst_is_device && !stage) pool_free(d, M->stream);
        if (e != cudaSuccess) return cuda_fail(e, "download coordinates");
        return SLS_OK;
    }
    if (M->f32) {
        const float *f = reinterpret_cast<const float *>(src);
        if (dst_is_device) {
            SLS_CUDA_TRY(launch_widen(f, xy_out, M->n, M->opt.layout, device_sm_count() * 4, M->stream), "widen");
        } else {
            std::vector<float> tmp(2 * (size_t)M->n);
            SLS_CUDA_TRY(cudaMemcpyAsync(tmp.data(), f, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost,
                                         M->stream), "download");
            SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "download");
            for (int64_t i = 0; i < M->n; ++i) {
                const bool soa = M->opt.layout == 1;
                xy_out[2 * i] = (double)tmp[soa ? i : 2 * i];
                xy_out[2 * i + 1] = (double)tmp[soa ? M->n + i : 2 * i + 1];
            }
        }
    } else if (M->opt.layout == 0) {
        SLS_CUDA_TRY(cudaMemcpyAsync(xy_out, src, cbytes,
                                     dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     M->stream), "download coordinates");
    } else if (dst_is_device) {
        SLS_CUDA_TRY(launch_soa_to_aos(src, xy_out, M->n, device_sm_count() * 4, M->stream), "interleave");
    } else {
        std::vector<double> tmp(2 * M->n);
        SLS_CUDA_TRY(cudaMemcpyAsync(tmp.data(), src, cbytes, cudaMemcpyDeviceToHost, M->stream), "download");
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "download");
        for (int64_t i = 0; i < M->n; ++i) {
            xy_out[2 * i] = tmp[i];
            xy_out[2 * i + 1] = tmp[M->n + i];
        }
    }
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "download coordinates");
    return SLS_OK;
}

sls_status mesh_set_coords(sls_mesh *M, const double *xy, bool src_is_device)
{
    if (M->perm) {
        // renumbered mesh: into the mesh's numbering (and layout, and type) on the device
        const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
        const size_t ebytes = (M->f32 ? sizeof(float) : sizeof(double)) * 2 * (size_t)M->n;
        double *d = const_cast<double *>(xy);
        sls_status st;
        if (!src_is_device && (st = dev_alloc(M, (void **)&d, cbytes, "upload")) != SLS_OK) return st;
        cudaError_t e = cudaSuccess;
        if (!src_is_device) e = cudaMemcpyAsync(d, xy, cbytes, cudaMemcpyHostToDevice, M->stream);
        if (e == cudaSuccess)
            e = launch_permute_from_aos(d, M->opt.layout, M->f32, M->n, M->perm, M->xy[M->cur],
                                        device_sm_count() * 4, M->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(M->xy[M->cur ^ 1], M->xy[M->cur], ebytes, cudaMemcpyDeviceToDevice, M->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
        if (!src_is_device) pool_free(d, M->stream);
        if (e != cudaSuccess) return cuda_fail(e, "set coordinates");
        return SLS_OK;
    }
    if (M->f32) {
        const size_t fbytes = sizeof(float) * 2 * (size_t)M->n;
        float *f = reinterpret_cast<float *>(M->xy[M->cur]);
        if (src_is_device) {
            SLS_CUDA_TRY(launch_narrow(xy, f, M->n, M->opt.layout, device_sm_count() * 4, M->stream), "narrow");
        } else {
            std::vector<float> tmp(2 * (size_t)M->n);
            for (int64_t i = 0; i < M->n; ++i) {
                const bool soa = M->opt.layout == 1;
                tmp[soa ? i : 2 * i] = (float)xy[2 * i];
                tmp[soa ? M->n + i : 2 * i + 1] = (float)xy[2 * i + 1];
            }
            SLS_CUDA_TRY(cudaMemcpyAsync(f, tmp.data(), fbytes, cudaMemcpyHostToDevice, M->stream), "upload");
            SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "upload");
        }
        SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[M->cur ^ 1], f, fbytes, cudaMemcpyDeviceToDevice, M->stream), "copy");
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "set coordinates");
        return SLS_OK;
    }
    const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
    if (src_is_device) {
        if (M->opt.layout == 0)
            SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[M->cur], xy, cbytes, cudaMemcpyDeviceToDevice, M->stream), "copy");
        else
            SLS_CUDA_TRY(launch_aos_to_soa(xy, M->xy[M->cur], M->n, device_sm_count() * 4, M->stream), "split");
    } else {
        std::vector<double> tmp;
        const double *src = xy;
        if (M->opt.layout == 1) {
            to_soa(xy, M->n, tmp);
            src = tmp.data();
        }
        SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[M->cur], src, cbytes, cudaMemcpyHostToDevice, M->stream), "upload");
        SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "upload");
    }
    SLS_CUDA_TRY(cudaMemcpyAsync(M->xy[M->cur ^ 1], M->xy[M->cur], cbytes, cudaMemcpyDeviceToDevice,
                                 M->stream), "copy");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "set coordinates");
    return SLS_OK;
}

sls_status mesh_transfer_nodes(sls_mesh *M, const int32_t *idx, int64_t k, double *buf, bool scatter)
{
    if (M->f32) return fail(SLS_ERR_INVALID, "node gather/scatter needs an FP64 mesh");
    if (M->opt.form != 0) return fail(SLS_ERR_INVALID, "node gather/scatter needs a Form-A mesh");
    if (k == 0) return SLS_OK;
    if (!M->xfer_bad) {
        sls_status st = dev_alloc(M, (void **)&M->xfer_bad, sizeof(unsigned), "transfer flag");
        if (st != SLS_OK) return st;
    }
    const int grid = device_sm_count() * 4;
    SLS_CUDA_TRY(cudaMemsetAsync(M->xfer_bad, 0, sizeof(unsigned), M->stream), "transfer");
    if (scatter)
        SLS_CUDA_TRY(launch_scatter_nodes(M->xy[0], M->xy[1], M->opt.layout, M->n, idx, k, M->inv, buf,
                                          M->xfer_bad, grid, M->stream), "scatter");
    else
        SLS_CUDA_TRY(launch_gather_nodes(M->xy[M->cur], M->opt.layout, M->n, idx, k, M->inv, buf, M->xfer_bad,
                                         grid, M->stream), "gather");
    SLS_CUDA_TRY(cudaMemcpyAsync(M->h_stats, M->xfer_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, M->stream),
                 "transfer");
    SLS_CUDA_TRY(cudaStreamSynchronize(M->stream), "transfer");
    unsigned bad;
    std::memcpy(&bad, M->h_stats, sizeof bad);
    if (bad) return fail(SLS_ERR_INVALID, "a node id is outside [0, n)");
    return SLS_OK;
}

sls_status mesh_histogram(const sls_mesh *M, int nbins, double lo, double hi, int64_t *counts,
                          double *qmin, double *qmean)
{
    unsigned long long *d_counts = nullptr, *d_key = nullptr;
    double *d_sum = nullptr;
    sls_status st;
    // binary32 meshes: alpha (FP64) of the coordinates widened exactly
    double *wide = nullptr;
    const double *hx = M->xy[M->cur];
    int hlayout = M->opt.layout;
    if (M->f32) {
        if ((st = dev_alloc(M, (void **)&wide, sizeof(double) * 2 * (size_t)M->n, "histogram")) != SLS_OK) return st;
        cudaError_t e0 = launch_widen(reinterpret_cast<const float *>(M->xy[M->cur]), wide, M->n, M->opt.layout,
                                      device_sm_count() * 4, M->stream);
        if (e0 != cudaSuccess) {
            pool_free(wide, M->stream);
            return cuda_fail(e0, "widen");
        }
        hx = wide;
        hlayout = 0;
    }
    if ((st = dev_alloc(M, (void **)&d_counts, sizeof(unsigned long long) * (nbins + 2), "histogram")) != SLS_OK) {
        pool_free(wide, M->stream);
        return st;
    }
    d_key = d_counts + nbins;
    d_sum = reinterpret_cast<double *>(d_counts + nbins + 1);
    std::vector<unsigned long long> h(nbins + 2);
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(unsigned long long) * (nbins + 2), M->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_key, 0xff, sizeof(unsigned long long), M->stream);
    if (e == cudaSuccess)
        e = launch_histogram(hx, hlayout, M->n, M->tri, M->m, nbins, lo, hi, d_counts, d_key, d_sum,
                             device_sm_count() * 8, M->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_counts, sizeof(unsigned long long) * (nbins + 2),
                            cudaMemcpyDeviceToHost, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    pool_free(d_counts, M->stream);
    pool_free(wide, M->stream);
    if (e != cudaSuccess) return cuda_fail(e, "histogram");
    for (int b = 0; b < nbins; ++b) counts[b] = (int64_t)h[b];
    unsigned long long key = h[nbins];
    unsigned long long bits = (key >> 63) ? (key & 0x7fffffffffffffffull) : ~key;
    double mn, sum;
    std::memcpy(&mn, &bits, sizeof mn);
    std::memcpy(&sum, &h[nbins + 1], sizeof sum);
    if (qmin) *qmin = mn;
    if (qmean) *qmean = sum / (double)M->m;
    return SLS_OK;
}

}  // namespace sls
