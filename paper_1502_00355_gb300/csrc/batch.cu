// batch.cu -- the batched form: many meshes of uneven size smoothed together.
//
// The meshes keep their own device buffers (from sls_mesh_create); the batch
// adds a job table (one JobDesc per mesh), a list of warp tasks (32 nodes of
// one mesh each) ordered by descending iteration count, and one statistics
// record per mesh and pass.  Round r runs pass r of every mesh that still
// has passes left; the rounds of a whole sls_batch_smooth call are captured
// once into a CUDA graph and replayed with a single cudaGraphLaunch.  Every
// mesh gets exactly the arithmetic of sls_smooth, so results are
// bit-identical to smoothing it alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "api_common.h"
#include "kernels.h"

using namespace sls;

struct sls_batch {
    std::vector<sls_mesh *> meshes;
    std::vector<int32_t> iters;
    std::vector<double> tols;
    std::vector<int> order;            // job slot -> mesh index (descending iterations)
    int layout = 0, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    JobDesc *d_jobs = nullptr;
    JobDesc *h_jobs = nullptr;         // pinned staging of the job table
    WarpTask *d_tasks = nullptr;
    int64_t ntasks = 0;
    std::vector<int64_t> round_tasks;  // tasks taking part in round r
    PassStats *d_stats = nullptr;
    std::vector<int64_t> stats_off;    // per job slot
    int64_t nstats = 0;
    std::vector<double *> d_start;     // per mesh: the packed starting coordinates
    int rounds = 0;
    int block = 128, grid = 0;
    int64_t chunk = 0;                 // tasks per warp chunk (launch_batch_pass)
    unsigned long long *d_claim = nullptr;  // one chunk counter per round (dynamic chunks)
    cudaGraphExec_t exec = nullptr;
};

namespace {

#define BATCH_TRY(expr, what)                              \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

void release(sls_batch *B)
{
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->exec) cudaGraphExecDestroy(B->exec);
    cudaFree(B->d_jobs);
    cudaFree(B->d_tasks);
    cudaFree(B->d_stats);
    cudaFree(B->d_claim);
    if (B->h_jobs) cudaFreeHost(B->h_jobs);
    for (double *p : B->d_start) cudaFree(p);
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    B->stream = nullptr;
}

sls_status build_graph(sls_batch *B)
{
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    BATCH_TRY(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t err = cudaSuccess;
    for (int r = 0; r < B->rounds && err == cudaSuccess; ++r)
        err = launch_batch_pass(B->d_jobs, B->d_tasks, B->round_tasks[r], r, B->layout, B->block, B->grid,
                                B->stream, B->chunk, B->d_claim + r);
    cudaError_t e2 = cudaStreamEndCapture(B->stream, &g);
    if (err != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(err, "capture batch rounds");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    err = cudaGraphInstantiate(&B->exec, g, 0);
    cudaGraphDestroy(g);
    if (err != cudaSuccess) return cuda_fail(err, "instantiate batch graph");
    return SLS_OK;
}

sls_status run(sls_batch *B, sls_info *infos)
{
    const int k = (int)B->meshes.size();
    for (int slot = 0; slot < k; ++slot) {
        const int mi = B->order[slot];
        sls_mesh *M = B->meshes[mi];
        JobDesc &J = B->h_jobs[slot];
        J.xy[0] = M->xy[0];
        J.xy[1] = M->xy[1];
        J.node_off = M->node_off;
        J.adj = M->adj;
        J.n = M->n;
        J.stats = B->d_stats + B->stats_off[slot];
        const double tol = B->tols[mi];
        const double thr = tolerance_threshold(tol, M->diag);
        std::memcpy(&J.thr_bits, &thr, sizeof thr);
        J.strict = M->opt.accept_strict;
        J.tol_active = tol > 0.0 ? 1 : 0;
        J.max_iter = B->iters[mi];
        J.base_round = 0;
        J.cur0 = M->cur;
        J.pad = 0;
        J.accept = M->accept;
    }
    BATCH_TRY(cudaMemcpyAsync(B->d_jobs, B->h_jobs, sizeof(JobDesc) * k, cudaMemcpyHostToDevice, B->stream),
              "upload job table");
    BATCH_TRY(cudaMemsetAsync(B->d_stats, 0, sizeof(PassStats) * B->nstats, B->stream), "clear statistics");
    BATCH_TRY(cudaMemsetAsync(B->d_claim, 0, sizeof(unsigned long long) * std::max(1, B->rounds), B->stream),
              "clear chunk counters");
    if (B->rounds > 0) {
        if (!B->exec) {
            sls_status st = build_graph(B);
            if (st != SLS_OK) return st;
        }
        BATCH_TRY(cudaGraphLaunch(B->exec, B->stream), "launch batch graph");
    }
    std::vector<PassStats> hs(B->nstats);
    BATCH_TRY(cudaMemcpyAsync(hs.data(), B->d_stats, sizeof(PassStats) * B->nstats, cudaMemcpyDeviceToHost,
                              B->stream), "read statistics");
    BATCH_TRY(cudaStreamSynchronize(B->stream), "batch smooth");
    for (int slot = 0; slot < k; ++slot) {
        const int mi = B->order[slot];
        sls_mesh *M = B->meshes[mi];
        const PassStats *st = hs.data() + B->stats_off[slot];
        sls_info info{};
        int it = 0;
        long long fb = 0;
        while (it < B->iters[mi] && st[it].executed) fb += (long long)st[it++].fallbacks;
        info.iterations = it;
        info.fp64_fallbacks = fb;
        if (it > 0) {
            const double tol = B->tols[mi];
            const double thr = tolerance_threshold(tol, M->diag);
            unsigned long long thr_bits;
            std::memcpy(&thr_bits, &thr, sizeof thr);
            info.accepted_last = (int64_t)st[it - 1].nacc;
            std::memcpy(&info.max_d2_last, &st[it - 1].maxd2_bits, sizeof(double));
            info.converged = (tol > 0.0 && st[it - 1].maxd2_bits < thr_bits) ? 1 : 0;
        }
        M->cur ^= (it & 1);
        M->last = info;
        if (infos) infos[mi] = info;
    }
    return SLS_OK;
}

sls_status reset(sls_batch *B)
{
    for (size_t mi = 0; mi < B->meshes.size(); ++mi) {
        sls_mesh *M = B->meshes[mi];
        const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
        BATCH_TRY(cudaMemcpyAsync(M->xy[0], B->d_start[mi], cbytes, cudaMemcpyDeviceToDevice, B->stream), "reset");
        BATCH_TRY(cudaMemcpyAsync(M->xy[1], B->d_start[mi], cbytes, cudaMemcpyDeviceToDevice, B->stream), "reset");
        M->cur = 0;
    }
    BATCH_TRY(cudaStreamSynchronize(B->stream), "reset");
    return SLS_OK;
}

// Picks the launch shape by timing a whole batch smooth for each candidate,
// restoring the starting coordinates after every trial: the block size (32-
// node tasks a CTA runs at once, 4 per 128 threads) and the chunk of
// consecutive tasks a warp takes: one contiguous share of the list (0), 64
// in a grid stride, or 32 claimed from a per-round counter.  Every round of a call is one node of one
// CUDA graph, so all passes of a call are one launch whatever the shape.
sls_status autotune(sls_batch *B, bool tune_block)
{
    struct Shape {
        int block;
        int64_t chunk;
    };
    std::vector<Shape> cands;
    const int blocks[2] = {64, 128};  // the kernel is built for 6 blocks of <= 128
    // chunks of 1 to 16 tasks measured 11-60% slower on the 2,048-mesh
    // workload: a warp that changes job drains its deferred nodes at partial
    // width, so short chunks run the exact FP64 path with few lanes active
    const int64_t chunks[3] = {0, 64, -32};  // < 0: claimed from a per-round counter
    for (int b : blocks) {
        if (!tune_block && b != B->block) continue;
        for (int64_t c : chunks) cands.push_back(Shape{b, c});
    }
    if (cands.empty())
        for (int64_t c : chunks) cands.push_back(Shape{B->block, c});
    float best_ms = -1.0f;
    Shape best = cands[0];
    cudaEvent_t e0, e1;
    BATCH_TRY(cudaEventCreate(&e0), "event");
    BATCH_TRY(cudaEventCreate(&e1), "event");
    sls_status st = SLS_OK;
    for (size_t c = 0; c < cands.size() && st == SLS_OK; ++c) {
        B->block = cands[c].block;
        B->chunk = cands[c].chunk;
        B->grid = device_sm_count() * batch_pass_occupancy(B->layout, B->block);
        if (B->rounds > 0) st = build_graph(B);
        if (st != SLS_OK) break;
        cudaEventRecord(e0, B->stream);
        st = run(B, nullptr);
        cudaEventRecord(e1, B->stream);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == SLS_OK && (best_ms < 0.0f || ms < best_ms)) {
            best_ms = ms;
            best = cands[c];
        }
        if (st == SLS_OK) st = reset(B);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SLS_OK) return st;
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    B->block = best.block;
    B->chunk = best.chunk;
    B->grid = device_sm_count() * batch_pass_occupancy(B->layout, B->block);
    return SLS_OK;
}

}  // namespace

extern "C" {

sls_status sls_batch_create(sls_mesh *const *meshes, int32_t k, const int32_t *iters, const double *tol_rel,
                            const sls_options *opt, sls_batch **out)
{
    if (!out) return fail(SLS_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (!meshes || !iters || k < 1) return fail(SLS_ERR_INVALID, "need k >= 1 meshes and their iteration counts");
    int dev = 0;
    BATCH_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    for (int j = 0; j < k; ++j) {
        if (!meshes[j]) return fail(SLS_ERR_INVALID, "mesh handle is NULL");
        if (meshes[j]->device != dev) return fail(SLS_ERR_INVALID, "all meshes must live on the current device");
        if (meshes[j]->opt.layout != meshes[0]->opt.layout)
            return fail(SLS_ERR_INVALID, "all meshes of a batch must use the same layout");
        if (meshes[j]->opt.form != 0 || meshes[j]->f32)
            return fail(SLS_ERR_INVALID, "the batched form runs FP64 Form A meshes only");
        if (iters[j] < 0) return fail(SLS_ERR_INVALID, "iteration counts must be >= 0");
        if (tol_rel && std::isnan(tol_rel[j])) return fail(SLS_ERR_INVALID, "tolerance is NaN");
        for (int i = 0; i < j; ++i)
            if (meshes[i] == meshes[j]) return fail(SLS_ERR_INVALID, "a mesh appears twice in the batch");
    }
    sls_options o = resolve_options(opt);
    sls_batch *B = new (std::nothrow) sls_batch();
    if (!B) return fail(SLS_ERR_OOM, "host allocation failed");
    B->meshes.assign(meshes, meshes + k);
    B->iters.assign(iters, iters + k);
    B->tols.assign(k, 0.0);
    if (tol_rel) B->tols.assign(tol_rel, tol_rel + k);
    B->layout = meshes[0]->opt.layout;
    B->device = dev;
    auto fail_free = [B](sls_status st) {
        release(B);
        delete B;
        return st;
    };
    if (o.stream) {
        B->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail_free(fail(SLS_ERR_CUDA, "cudaStreamCreate"));
        B->own_stream = true;
    }
    B->order.resize(k);
    std::iota(B->order.begin(), B->order.end(), 0);
    std::stable_sort(B->order.begin(), B->order.end(), [B](int a, int b) { return B->iters[a] > B->iters[b]; });
    std::vector<WarpTask> tasks;
    std::vector<int64_t> tasks_upto(k + 1, 0);
    B->stats_off.resize(k);
    for (int slot = 0; slot < k; ++slot) {
        sls_mesh *M = B->meshes[B->order[slot]];
        for (int64_t f = 0; f < M->n; f += 32) tasks.push_back(WarpTask{slot, (int32_t)f});
        tasks_upto[slot + 1] = (int64_t)tasks.size();
        B->stats_off[slot] = B->nstats;
        B->nstats += std::max(1, B->iters[B->order[slot]]);
    }
    B->ntasks = (int64_t)tasks.size();
    B->rounds = B->iters[B->order[0]];
    B->round_tasks.assign(B->rounds, 0);
    for (int r = 0; r < B->rounds; ++r) {
        int slots = 0;
        while (slots < k && B->iters[B->order[slots]] > r) ++slots;
        B->round_tasks[r] = tasks_upto[slots];
    }
    if (cudaMalloc(&B->d_jobs, sizeof(JobDesc) * k) != cudaSuccess ||
        cudaMalloc(&B->d_tasks, sizeof(WarpTask) * std::max<int64_t>(1, B->ntasks)) != cudaSuccess ||
        cudaMalloc(&B->d_stats, sizeof(PassStats) * B->nstats) != cudaSuccess ||
        cudaMalloc(&B->d_claim, sizeof(unsigned long long) * std::max(1, B->rounds)) != cudaSuccess ||
        cudaMallocHost(&B->h_jobs, sizeof(JobDesc) * k) != cudaSuccess) {
        cudaGetLastError();
        return fail_free(fail(SLS_ERR_OOM, "batch allocation failed"));
    }
    if (cudaMemcpy(B->d_tasks, tasks.data(), sizeof(WarpTask) * B->ntasks, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail_free(fail(SLS_ERR_CUDA, "upload warp tasks"));
    B->d_start.assign(k, nullptr);
    for (int j = 0; j < k; ++j) {
        sls_mesh *M = B->meshes[j];
        const size_t cbytes = sizeof(double) * 2 * (size_t)M->n;
        if (cudaMalloc(&B->d_start[j], cbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail_free(fail(SLS_ERR_OOM, "batch allocation failed"));
        }
        if (cudaMemcpyAsync(B->d_start[j], M->xy[M->cur], cbytes, cudaMemcpyDeviceToDevice, B->stream) != cudaSuccess)
            return fail_free(fail(SLS_ERR_CUDA, "save starting coordinates"));
    }
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return fail_free(fail(SLS_ERR_CUDA, "batch set-up"));
    if (opt != nullptr && opt->block_size > 0) {
        if (opt->block_size < 32 || opt->block_size > 128)
            return fail_free(fail(SLS_ERR_INVALID, "batch block_size must be 32, 64, 96 or 128"));
        B->block = opt->block_size;
    }
    B->grid = device_sm_count() * batch_pass_occupancy(B->layout, B->block);
    {
        // autotune on the packed meshes (the block size too unless it was
        // given), then restore their coordinates
        sls_status st = autotune(B, opt == nullptr || opt->block_size == 0);
        if (st != SLS_OK) return fail_free(st);
    }
    *out = B;
    return SLS_OK;
}

sls_status sls_batch_smooth(sls_batch *B, sls_info *infos)
{
    if (!B) return fail(SLS_ERR_INVALID, "batch must not be NULL");
    return run(B, infos);
}

sls_status sls_batch_get_coords(const sls_batch *B, int32_t j, double *xy_out)
{
    if (!B || !xy_out) return fail(SLS_ERR_INVALID, "batch and xy_out must not be NULL");
    if (j < 0 || j >= (int32_t)B->meshes.size()) return fail(SLS_ERR_INVALID, "mesh index out of range");
    return mesh_download(B->meshes[j], xy_out, false);
}

sls_status sls_batch_reset(sls_batch *B)
{
    if (!B) return fail(SLS_ERR_INVALID, "batch must not be NULL");
    return reset(B);
}

sls_status sls_batch_shape(const sls_batch *B, int32_t *block, int64_t *chunk)
{
    if (!B) return fail(SLS_ERR_INVALID, "batch must not be NULL");
    if (block) *block = B->block;
    if (chunk) *chunk = B->chunk;
    return SLS_OK;
}

sls_status sls_batch_set_shape(sls_batch *B, int32_t block, int64_t chunk)
{
    if (!B) return fail(SLS_ERR_INVALID, "batch must not be NULL");
    if (block != 32 && block != 64 && block != 96 && block != 128)
        return fail(SLS_ERR_INVALID, "batch block size must be 32, 64, 96 or 128");
    if (chunk < -(int64_t(1) << 20) || chunk > (int64_t(1) << 20)) return fail(SLS_ERR_INVALID, "chunk out of range");
    if (B->exec) {
        cudaGraphExecDestroy(B->exec);
        B->exec = nullptr;
    }
    B->block = block;
    B->chunk = chunk;
    B->grid = device_sm_count() * batch_pass_occupancy(B->layout, B->block);
    return SLS_OK;
}

sls_status sls_batch_destroy(sls_batch *B)
{
    if (!B) return SLS_OK;
    release(B);
    delete B;
    return SLS_OK;
}

}  // extern "C"
