// noalloc.cu -- sls_smooth_noalloc: smoothing passes that allocate nothing.
//
// Some callers cannot allocate device memory at the point where they smooth:
// latency-critical loops that must not hit the implicit device
// synchronisation of cudaMalloc/cudaFree, plug-ins whose host application
// owns the whole device memory budget through its own pool, and services
// that fix their memory at start-up and must not fail for lack of it later.
// This entry point runs the same pass kernels as sls_smooth, on two
// coordinate buffers the caller already owns, and keeps the only scratch the
// kernels need -- one statistics record per pass -- in a fixed array in
// device global memory that is part of the library image.
#include <cmath>
#include <cstring>
#include <mutex>

#include "api_common.h"
#include "kernels.h"

namespace sls {
namespace {

// Scratch: one statistics record per pass, 4096 passes (128 KiB).  Every GPU
// that loads the library holds one copy until the process exits.  All calls
// on a device share it, so calls whose work overlaps on the GPU race.
constexpr int kNoAllocMaxPasses = SLS_NOALLOC_MAX_PASSES;
__device__ __align__(256) PassStats g_noalloc_stats[kNoAllocMaxPasses];

// Host code may not use g_noalloc_stats as an address: it is a host-side
// stand-in.  The device address is looked up with the device current and
// cached per device together with the context it belongs to; a new context
// on the device (after cudaDeviceReset) looks it up again.
constexpr int kMaxDevices = 64;
struct StatsAddr {
    unsigned long long ctx = 0ull;
    PassStats *ptr = nullptr;
};
StatsAddr g_stats_addr[kMaxDevices];
std::mutex g_setup_mu;

sls_status stats_address(PassStats **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SLS_ERR_INVALID, "device ordinal out of range");
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mu);
    StatsAddr &c = g_stats_addr[dev];
    if (!c.ptr || ctx == 0ull || c.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_stats);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the pass statistics");
        c.ptr = static_cast<PassStats *>(p);
        c.ctx = ctx;
    }
    *out = c.ptr;
    return SLS_OK;
}

}  // namespace

// Called by sls_mesh_create, which allocates anyway: looking the array up
// loads this file's device code and data on the device (CUDA loads modules
// lazily), so a later sls_smooth_noalloc on the mesh finds it in place.
sls_status noalloc_prepare()
{
    PassStats *p = nullptr;
    return stats_address(&p);
}

}  // namespace sls

using namespace sls;

extern "C" sls_status sls_smooth_noalloc(const sls_mesh *M, double *xy_in, double *xy_out,
                                         int32_t max_iter, double tol_rel, void *stream,
                                         sls_info *info)
{
    if (!M || !xy_in || !xy_out) return fail(SLS_ERR_INVALID, "mesh, xy_in and xy_out must not be NULL");
    if (xy_in == xy_out) return fail(SLS_ERR_INVALID, "xy_in and xy_out must be distinct buffers");
    if (M->opt.layout != 0) return fail(SLS_ERR_INVALID, "sls_smooth_noalloc needs a mesh with the AoS layout");
    if (M->opt.form != 0 || M->f32) return fail(SLS_ERR_INVALID, "sls_smooth_noalloc runs FP64 Form A only");
    if (max_iter < 0 || max_iter > kNoAllocMaxPasses)
        return fail(SLS_ERR_INVALID, "max_iter must be in [0, SLS_NOALLOC_MAX_PASSES] for sls_smooth_noalloc");
    if (std::isnan(tol_rel)) return fail(SLS_ERR_INVALID, "tol_rel is NaN");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != M->device) return fail(SLS_ERR_INVALID, "the mesh's device must be the current device");
    PassStats *stats = nullptr;
    sls_status st = stats_address(&stats);
    if (st != SLS_OK) return st;
    cudaStream_t s = stream ? (cudaStream_t)stream : M->stream;
    const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;

    sls_info res{};
    if (max_iter > 0) {
        e = cudaMemsetAsync(stats, 0, sizeof(PassStats) * (size_t)max_iter, s);
        if (e != cudaSuccess) return cuda_fail(e, "clear the pass statistics");
        if (M->perm) {
            // a mesh renumbered inside the library: the start into its numbering
            e = launch_permute_coords(xy_in, xy_out, 0, false, M->n, M->perm, device_sm_count() * 4, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(xy_in, xy_out, cbytes, cudaMemcpyDeviceToDevice, s);
        } else {
            // passes never write fixed nodes, so both buffers must start equal
            e = cudaMemcpyAsync(xy_out, xy_in, cbytes, cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "copy the starting coordinates");
    }
    const bool tol_active = tol_rel > 0.0;
    const double thr = tolerance_threshold(tol_rel, M->diag);
    unsigned long long thr_bits;
    std::memcpy(&thr_bits, &thr, sizeof thr_bits);
    PassArgs a{};
    a.node_off = M->node_off;
    a.adj = M->adj;
    a.n = M->n;
    a.order = nullptr;
    a.norder = 0;
    a.stats = stats;
    a.strict = M->opt.accept_strict;
    a.tol_active = tol_active ? 1 : 0;
    a.thr_bits = thr_bits;
    a.accept = nullptr;
    double *buf[2] = {xy_in, xy_out};
    PassStats probe;
    int launched = 0;
    while (launched < max_iter) {
        const int end = launched + M->opt.passes_per_check < max_iter ? launched + M->opt.passes_per_check
                                                                      : max_iter;
        for (int q = launched; q < end; ++q) {
            a.in = buf[q & 1];
            a.out = buf[(q + 1) & 1];
            a.q = q;
            e = M->screened ? launch_pass_screened(a, 0, M->block, M->grid, s)
                            : launch_pass_fp64(a, 0, M->block, M->grid, s);
            if (e != cudaSuccess) return cuda_fail(e, "pass kernel");
        }
        launched = end;
        if (tol_active && launched < max_iter) {
            e = cudaMemcpyAsync(&probe, stats + launched - 1, sizeof probe, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return cuda_fail(e, "read pass statistics");
            if (probe.executed == 0u || probe.maxd2_bits < thr_bits) break;
        }
    }
    // executed passes form a prefix; read them back in small stack-sized pieces
    int it = 0;
    long long fb = 0;
    PassStats last{};
    PassStats chunk[32];
    for (int q0 = 0; q0 < launched && it == q0; q0 += 32) {
        const int cnt = launched - q0 < 32 ? launched - q0 : 32;
        e = cudaMemcpyAsync(chunk, stats + q0, sizeof(PassStats) * cnt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "read pass statistics");
        for (int k = 0; k < cnt && chunk[k].executed; ++k) {
            fb += (long long)chunk[k].fallbacks;
            last = chunk[k];
            ++it;
        }
    }
    // the result of pass it-1 is in buf[it & 1]; make xy_out hold it (in the
    // caller's numbering: a renumbered mesh's result goes back through xy_in)
    if (M->perm && max_iter > 0) {
        e = (it & 1) ? cudaMemcpyAsync(xy_in, xy_out, cbytes, cudaMemcpyDeviceToDevice, s) : cudaSuccess;
        if (e == cudaSuccess)
            e = launch_unpermute_to_aos(xy_in, 0, false, M->n, M->perm, xy_out, device_sm_count() * 4, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "copy the result");
    } else if ((it & 1) == 0) {
        e = cudaMemcpyAsync(xy_out, xy_in, cbytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "copy the result");
    }
    res.iterations = it;
    res.fp64_fallbacks = fb;
    res.launches = launched;
    if (it > 0) {
        res.accepted_last = (int64_t)last.nacc;
        std::memcpy(&res.max_d2_last, &last.maxd2_bits, sizeof(double));
        res.converged = (tol_active && last.maxd2_bits < thr_bits) ? 1 : 0;
    }
    if (info) *info = res;
    return SLS_OK;
}
