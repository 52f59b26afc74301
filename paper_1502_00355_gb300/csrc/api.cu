// api.cu -- the single-mesh C ABI of slsmooth (see include/slsmooth.h).
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "api_common.h"
#include "kernels.h"

namespace sls {

thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

sls_status fail(sls_status code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

sls_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear a sticky launch error so the handle stays usable
    return fail(SLS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// The driver's cuCtxGetCurrent and cuCtxGetId, looked up through the runtime
// so the library does not link the driver library itself (it must load on
// machines without a GPU driver).
unsigned long long current_context_id()
{
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0ull;
    void *ctx = nullptr;
    unsigned long long id = 0ull;
    if (get_current(&ctx) != 0 || !ctx) return 0ull;
    if (get_id(ctx, &id) != 0) return 0ull;
    return id;
}

int device_sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

static sls_options g_defaults = {0, 0, 0, SLS_KERNEL_AUTO, 0, 0, 0, 16, 0, 0, 64, 0, 0, nullptr};

sls_options resolve_options(const sls_options *opt)
{
    sls_options o = opt ? *opt : g_defaults;
    if (o.block_size <= 0) o.block_size = 256;
    if (o.passes_per_check <= 0) o.passes_per_check = 16;
    if (o.precision == 0) o.precision = 64;
    return o;
}

sls_status check_options(const sls_options &o)
{
    if (o.layout != 0 && o.layout != 1) return fail(SLS_ERR_INVALID, "layout must be 0 (AoS) or 1 (SoA)");
    if (o.kernel < SLS_KERNEL_AUTO || o.kernel > SLS_KERNEL_FILTERED)
        return fail(SLS_ERR_INVALID, "unknown kernel");
    if (o.block_size % 32 != 0 || o.block_size > 1024)
        return fail(SLS_ERR_INVALID, "block_size must be a multiple of 32, at most 1024");
    if (o.form != 0 && o.form != 1) return fail(SLS_ERR_INVALID, "form must be 0 (Form A) or 1 (Form B)");
    if (o.precision != 32 && o.precision != 64) return fail(SLS_ERR_INVALID, "precision must be 32 or 64");
    if (o.skip_unchanged != 0 && o.skip_unchanged != 1) return fail(SLS_ERR_INVALID, "skip_unchanged must be 0 or 1");
    if (o.numbering < 0 || o.numbering > 2) return fail(SLS_ERR_INVALID, "numbering must be 0, 1 or 2");
    if (o.skip_unchanged && (o.form != 0 || o.precision != 64 || o.kernel == SLS_KERNEL_FP64))
        return fail(SLS_ERR_INVALID, "skip_unchanged needs Form A, FP64 and the screened kernel");
    return SLS_OK;
}

}  // namespace sls

using namespace sls;

extern "C" {

void sls_default_options(sls_options *opt)
{
    if (opt) *opt = g_defaults;
}

const char *sls_status_str(sls_status s)
{
    switch (s) {
    case SLS_OK: return "ok";
    case SLS_ERR_INVALID: return "invalid argument or mesh";
    case SLS_ERR_NONMANIFOLD: return "non-manifold edge";
    case SLS_ERR_OOM: return "out of memory";
    case SLS_ERR_CUDA: return "CUDA error";
    case SLS_ERR_TIMEOUT: return "timed out";
    case SLS_ERR_BUSY: return "queue full";
    case SLS_ERR_REJECTED: return "job larger than the memory budget";
    case SLS_ERR_NOT_FOUND: return "unknown job";
    }
    return "unknown status";
}

const char *sls_last_error(void) { return g_last_error.c_str(); }

sls_status sls_mesh_create(const double *xy, int64_t n, const int32_t *tri, int64_t m,
                           const uint8_t *boundary, const sls_options *opt, sls_mesh **out)
{
    if (!out) return fail(SLS_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    sls_options o = resolve_options(opt);
    sls_status st = check_options(o);
    if (st != SLS_OK) return st;
    if (!xy || !tri) return fail(SLS_ERR_INVALID, "xy and tri must not be NULL");
    if (n < 3) return fail(SLS_ERR_INVALID, "a mesh needs at least 3 nodes");
    if (m < 1) return fail(SLS_ERR_INVALID, "a mesh needs at least 1 triangle");
    if (n >= (int64_t(1) << 31) || m >= (int64_t(1) << 31))
        return fail(SLS_ERR_INVALID, "n and m must be below 2^31");
    sls_mesh *M = new (std::nothrow) sls_mesh();
    if (!M) return fail(SLS_ERR_OOM, "host allocation failed");
    if (o.host_build) {
        HostMesh hm;
        st = build_host_mesh(xy, n, tri, m, boundary, hm);
        if (st == SLS_OK) st = mesh_upload(M, hm, xy, tri, o);
    } else {
        st = mesh_create_on_device(M, xy, n, tri, m, boundary, o);
    }
    if (st != SLS_OK) {
        mesh_release(M);
        delete M;
        return st;
    }
    *out = M;
    return SLS_OK;
}

sls_status sls_mesh_destroy(sls_mesh *mesh)
{
    if (!mesh) return SLS_OK;
    mesh_release(mesh);
    delete mesh;
    return SLS_OK;
}

sls_status sls_mesh_stats(const sls_mesh *M, int64_t *n, int64_t *m, int64_t *n_free, double *diag)
{
    if (!M) return fail(SLS_ERR_INVALID, "mesh must not be NULL");
    if (n) *n = M->n;
    if (m) *m = M->m;
    if (n_free) *n_free = M->n_free;
    if (diag) *diag = M->diag;
    return SLS_OK;
}

sls_status sls_smooth(sls_mesh *M, int32_t max_iter, double tol_rel, sls_info *info)
{
    if (!M) return fail(SLS_ERR_INVALID, "mesh must not be NULL");
    if (max_iter < 0) return fail(SLS_ERR_INVALID, "max_iter must be >= 0");
    if (std::isnan(tol_rel)) return fail(SLS_ERR_INVALID, "tol_rel is NaN");
    sls_info res{};
    sls_status st = mesh_run(M, max_iter, tol_rel, res);
    if (st != SLS_OK) return st;
    M->last = res;
    if (info) *info = res;
    return SLS_OK;
}

sls_status sls_get_coords(const sls_mesh *M, double *xy_out, int32_t dst_is_device)
{
    if (!M || !xy_out) return fail(SLS_ERR_INVALID, "mesh and xy_out must not be NULL");
    return mesh_download(M, xy_out, dst_is_device != 0);
}

sls_status sls_set_coords(sls_mesh *M, const double *xy, int32_t src_is_device)
{
    if (!M || !xy) return fail(SLS_ERR_INVALID, "mesh and xy must not be NULL");
    if (!src_is_device)
        for (int64_t k = 0; k < 2 * M->n; ++k)
            if (!std::isfinite(xy[k])) return fail(SLS_ERR_INVALID, "coordinates must be finite");
    return mesh_set_coords(M, xy, src_is_device != 0);
}

sls_status sls_gather_coords(sls_mesh *M, const int32_t *idx, int64_t k, double *out)
{
    if (!M) return fail(SLS_ERR_INVALID, "mesh must not be NULL");
    if (k < 0 || (k > 0 && (!idx || !out))) return fail(SLS_ERR_INVALID, "need k >= 0 and device idx and out");
    return mesh_transfer_nodes(M, idx, k, out, false);
}

sls_status sls_scatter_coords(sls_mesh *M, const int32_t *idx, int64_t k, const double *in)
{
    if (!M) return fail(SLS_ERR_INVALID, "mesh must not be NULL");
    if (k < 0 || (k > 0 && (!idx || !in))) return fail(SLS_ERR_INVALID, "need k >= 0 and device idx and in");
    return mesh_transfer_nodes(M, idx, k, const_cast<double *>(in), true);
}

sls_status sls_get_accept(const sls_mesh *M, uint8_t *accept_out)
{
    if (!M || !accept_out) return fail(SLS_ERR_INVALID, "mesh and accept_out must not be NULL");
    if (!M->accept) return fail(SLS_ERR_INVALID, "the mesh was created without record_accept");
    if (M->perm) {  // renumbered mesh: back to the caller's numbering
        uint8_t *d = nullptr;
        cudaError_t e = pool_alloc((void **)&d, (size_t)M->n, M->stream);
        if (e == cudaSuccess) e = launch_unpermute_u8(M->accept, M->n, M->perm, d, device_sm_count() * 4, M->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(accept_out, d, (size_t)M->n, cudaMemcpyDeviceToHost, M->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
        pool_free(d, M->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sls_get_accept");
        return SLS_OK;
    }
    cudaError_t e = cudaMemcpyAsync(accept_out, M->accept, (size_t)M->n, cudaMemcpyDeviceToHost, M->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sls_get_accept");
    return SLS_OK;
}

sls_status sls_quality_histogram(const sls_mesh *M, int32_t nbins, double lo, double hi,
                                 int64_t *counts, double *qmin, double *qmean)
{
    if (!M || !counts) return fail(SLS_ERR_INVALID, "mesh and counts must not be NULL");
    if (nbins < 1 || nbins > 4096) return fail(SLS_ERR_INVALID, "nbins must be in [1, 4096]");
    if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi))
        return fail(SLS_ERR_INVALID, "need finite lo < hi");
    return mesh_histogram(M, nbins, lo, hi, counts, qmin, qmean);
}

}  // extern "C"
