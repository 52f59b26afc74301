// server.cu -- the served form: smoothing jobs arriving over time, run with
// continuous batching.
//
// sls_submit copies a job's inputs and queues it.  A scheduler thread admits
// queued jobs in arrival order while a bound on their device footprint
// (coordinates, adjacency, statistics and the build's scratch) fits the
// memory budget, and hands them to builder threads.  Each builder owns a
// stream: it uploads the job's coordinates and triangles and builds the
// adjacency on the device (validation, neighbour finding and constraints,
// Sections 3.3.2 and 3.3.3), with stream-ordered allocations so that nothing
// waits for the rounds running on the other streams; a mesh with a node in
// more than 32 triangles is built on the host instead.  The scheduler runs
// rounds: one launch of the batched pass kernel over every active job, each
// at its own pass index.  After each round it reads every active job's
// statistics record and hands the jobs that reached their iteration cap or
// tolerance to a retire thread, which copies their coordinates back and
// frees their memory while the next round runs; queued jobs take the freed
// budget as it returns.  Latency is measured from sls_submit to the moment
// the result is on the host.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <cstdlib>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_common.h"
#include "kernels.h"

using namespace sls;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kBuilders = 4;  // builder threads (and streams) per server (12 measured no faster)
// Warp tasks of a round: one contiguous share of the list per warp (short
// chunks make warps change job often, and every change drains the warp's
// deferred nodes at partial width; measured on the batched form).
constexpr int64_t kServerChunk = 0;

enum JobState { kQueued, kBuilding, kActive, kRetiring, kDone, kFailed };

// Page-locked host blocks for the jobs' inputs and results, kept for reuse.
// A copy between the device and page-locked memory is one DMA that needs no
// CPU staging, so builds upload and results come back without a builder or
// the retire thread copying through the driver's bounce buffers; pinning
// memory is slow, so freed blocks are cached (up to kPinnedKeep bytes) for
// later jobs of a similar size.  Blocks come in powers of two from 64 KiB.
// When the driver refuses to pin more, plain host memory serves instead.
class PinnedCache {
public:
    static constexpr size_t kPinnedKeep = size_t(4) << 30;

    struct Block {
        void *p = nullptr;
        size_t cap = 0;
        bool pinned = false;
    };

    Block get(size_t bytes)
    {
        size_t cap = size_t(1) << 16;
        while (cap < bytes) cap <<= 1;
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto it = free_.find(cap);
            if (it != free_.end()) {
                Block b{it->second, cap, true};
                free_.erase(it);
                kept_ -= cap;
                return b;
            }
        }
        Block b{nullptr, cap, false};
        if (cudaMallocHost(&b.p, cap) == cudaSuccess) {
            b.pinned = true;
        } else {
            cudaGetLastError();
            b.p = std::malloc(cap);
            if (!b.p) throw std::bad_alloc();
        }
        return b;
    }

    void put(Block &b)
    {
        if (!b.p) return;
        if (b.pinned) {
            std::unique_lock<std::mutex> lk(mu_);
            if (kept_ + b.cap <= kPinnedKeep) {
                free_.emplace(b.cap, b.p);
                kept_ += b.cap;
                b = Block{};
                return;
            }
            lk.unlock();
            cudaFreeHost(b.p);
        } else {
            std::free(b.p);
        }
        b = Block{};
    }

    ~PinnedCache()
    {
        for (auto &kv : free_) cudaFreeHost(kv.second);
    }

private:
    std::mutex mu_;
    std::multimap<size_t, void *> free_;
    size_t kept_ = 0;
};

struct ServerJob {
    uint64_t id = 0;
    // inputs (one page-locked block: coordinates, triangles, boundary flags),
    // released once the job is on the device
    std::shared_ptr<PinnedCache> cache;  // where the host blocks go back to
    PinnedCache::Block in;
    const double *xy = nullptr;
    const int32_t *tri = nullptr;
    const uint8_t *boundary = nullptr;  // NULL: derived from open edges
    cudaEvent_t in_done = nullptr;      // the uploads from `in` are complete
    int64_t n = 0, m = 0;
    double diag = 0.0;
    int32_t max_iter = 0;
    double tol = 0.0;
    size_t reserved = 0;   // budget held: the bound at admission, the exact footprint once built
    // device state (stream-ordered allocations)
    double *d_xy[2] = {nullptr, nullptr};
    uint32_t *d_off = nullptr, *d_adj = nullptr;
    uint32_t *d_perm = nullptr;  // grouped numbering: internal id -> the caller's id (NULL: none)
    PassStats *d_stats = nullptr;
    cudaStream_t build_stream = nullptr;  // the builder stream the memory was allocated on
    cudaEvent_t uploaded = nullptr;
    int upload_state = 0;  // 0 pending, 1 built (event recorded), 2 failed
    int base_round = 0;
    int iterations = 0;
    bool finished = false;                // scheduler thread only: handed to the retire thread
    cudaEvent_t free_after = nullptr;     // the retire thread waits for it before touching the job
    // result
    JobState state = kQueued;
    sls_status status = SLS_OK;
    std::string error;
    PinnedCache::Block result;  // 2n doubles once done
    sls_info info{};
    Clock::time_point t_submit, t_done;

    void release_inputs()
    {
        if (in_done) {
            cudaEventSynchronize(in_done);
            cudaEventDestroy(in_done);
            in_done = nullptr;
        }
        if (cache) cache->put(in);
        xy = nullptr;
        tri = nullptr;
        boundary = nullptr;
    }

    ~ServerJob()
    {
        release_inputs();
        if (cache) cache->put(result);
    }
};

}  // namespace

struct sls_server {
    sls_options opt{};
    std::shared_ptr<PinnedCache> pinned = std::make_shared<PinnedCache>();
    size_t budget = 0, used = 0;
    int32_t max_queue = 0;
    int device = 0;
    cudaStream_t stream = nullptr, retire_stream = nullptr;
    std::vector<cudaStream_t> build_streams;

    std::mutex mu;
    std::condition_variable cv_build, cv_sched, cv_done, cv_retire;
    std::deque<std::shared_ptr<ServerJob>> queued, to_build, to_retire;
    std::vector<std::shared_ptr<ServerJob>> uploading, active;
    std::unordered_map<uint64_t, std::shared_ptr<ServerJob>> jobs;
    uint64_t next_id = 1;
    int64_t holding = 0;  // jobs whose inputs are still on the host (submitted, not yet built)
    bool stop = false, retire_stop = false;
    int builders_live = 0;
    std::vector<std::thread> builders;
    std::thread sched, retirer;

    // job table and warp tasks of the active set; the host staging and the
    // round records are double-buffered by round parity, because round r+1
    // is launched before the records of round r are read
    JobDesc *d_jobs = nullptr, *h_jobs[2] = {nullptr, nullptr};
    int64_t *d_toff = nullptr, *h_toff[2] = {nullptr, nullptr};  // first task of each job
    WarpTask *d_tasks = nullptr;
    size_t jobs_cap = 0, jobs_hcap[2] = {0, 0}, toff_cap = 0, toff_hcap[2] = {0, 0}, tasks_cap = 0;
    PassStats *h_round[2] = {nullptr, nullptr};  // pinned: a round's record of each job it ran over
    PassStats *d_round[2] = {nullptr, nullptr};  // the same records gathered on the device
    size_t round_cap[2] = {0, 0}, dround_cap[2] = {0, 0};
    cudaEvent_t ev_start[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    int64_t ntasks = 0;
    int block = 256, grid = 0;
    int round = 0;

    // statistics
    std::vector<double> latency_ms;
    double busy_s = 0.0;
    double node_updates = 0.0;
    int64_t completed = 0;
    std::string sched_error;
};

namespace {

// Device bytes a job holds once built: two coordinate arrays, node offsets,
// adjacency words, the numbering map, one statistics record per pass.
size_t built_footprint(int64_t n, uint64_t adj_words, int32_t max_iter)
{
    return 2 * sizeof(double) * 2 * (size_t)n + sizeof(uint32_t) * (size_t)(n + 1) + sizeof(uint32_t) * adj_words +
           sizeof(uint32_t) * (size_t)n + sizeof(PassStats) * (size_t)std::max(1, max_iter);
}

// A bound on what a job holds while it is built: the built footprint with
// at most n + 9m adjacency words (a meta word per node; per corner of a
// triangle at most two neighbours and one triangle code), plus the build's
// scratch (triangles, incidences, neighbour candidates, counts and flags;
// the numbering's inverse map and new offsets).
size_t admission_bound(int64_t n, int64_t m, int32_t max_iter)
{
    return built_footprint(n, (uint64_t)(n + 9 * m), max_iter) + 26 * (size_t)n + 48 * (size_t)m + 65536;
}

void fail_job(sls_server *S, ServerJob &J, sls_status st, const std::string &msg)
{
    J.state = kFailed;
    J.status = st;
    J.error = msg;
    J.t_done = Clock::now();
    S->cv_done.notify_all();
}

void free_job_device(ServerJob &J, cudaStream_t s)
{
    for (void *p : {(void *)J.d_xy[0], (void *)J.d_xy[1], (void *)J.d_off, (void *)J.d_adj, (void *)J.d_perm,
                    (void *)J.d_stats})
        if (p) cudaFreeAsync(p, s);
    if (J.uploaded) cudaEventDestroy(J.uploaded);
    J.d_xy[0] = J.d_xy[1] = nullptr;
    J.d_off = J.d_adj = J.d_perm = nullptr;
    J.d_stats = nullptr;
    J.uploaded = nullptr;
}

// Uploads job J on stream s and builds its adjacency there.  On success the
// job's device state is complete once J.uploaded has fired; *footprint is
// what it holds.  On failure everything is freed behind the stream's work.
sls_status build_job(ServerJob &J, bool group, cudaStream_t s, size_t *footprint)
{
    const int64_t n = J.n, m = J.m;
    const size_t cbytes = sizeof(double) * 2 * (size_t)n;
    int32_t *d_tri = nullptr;
    auto cleanup = [&](sls_status st) {
        if (d_tri) cudaFreeAsync(d_tri, s);
        free_job_device(J, s);
        return st;
    };
    auto cuda_err = [&](cudaError_t e, const char *what) { return cleanup(cuda_fail(e, what)); };
    cudaError_t e = cudaSuccess;
    for (void **p : {(void **)&J.d_xy[0], (void **)&J.d_xy[1]})
        if (e == cudaSuccess) e = pool_alloc(p, cbytes, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&d_tri, sizeof(int32_t) * 3 * (size_t)m, s);
    if (e == cudaSuccess) e = pool_alloc((void **)&J.d_stats, sizeof(PassStats) * (size_t)std::max(1, J.max_iter), s);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return cleanup(fail(SLS_ERR_OOM, "device allocation failed"));
    }
    if (e != cudaSuccess) return cuda_err(e, "device allocation");
    e = cudaMemcpyAsync(J.d_xy[0], J.xy, cbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_tri, J.tri, sizeof(int32_t) * 3 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&J.in_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(J.in_done, s);
    if (e != cudaSuccess) return cuda_err(e, "upload");
    DeviceAdjacency da;
    sls_status st = build_device_adjacency(n, m, J.d_xy[0], d_tri, J.boundary, true, s, da);
    if (st == SLS_ERR_NOT_FOUND) {
        // a node in more triangles than the device build handles: host build
        HostMesh hm;
        st = build_host_mesh(J.xy, n, J.tri, m, J.boundary, hm, 1);
        if (st != SLS_OK) return cleanup(st);
        da.adj_words = hm.node_off[n];
        da.n_free = hm.n_free;
        da.diag = hm.diag;
        e = pool_alloc((void **)&da.node_off, sizeof(uint32_t) * (size_t)(n + 1), s);
        if (e == cudaSuccess) e = pool_alloc((void **)&da.adj, sizeof(uint32_t) * std::max<uint64_t>(1, da.adj_words), s);
        J.d_off = da.node_off;  // freed with the job on any failure below
        J.d_adj = da.adj;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(da.node_off, hm.node_off.data(), sizeof(uint32_t) * (size_t)(n + 1),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(da.adj, hm.adj.data(), sizeof(uint32_t) * da.adj_words, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
        if (e != cudaSuccess) return cuda_err(e, "upload adjacency");
    } else if (st != SLS_OK) {
        return cleanup(st);
    }
    J.d_off = da.node_off;
    J.d_adj = da.adj;
    J.diag = da.diag;
    e = cudaFreeAsync(d_tri, s);
    d_tri = nullptr;
    if (e != cudaSuccess) return cuda_err(e, "build");
    if (group) {
        // Form A's grouped numbering (as for a single mesh): the coordinates
        // move to the new ids; the result goes back at retirement
        st = group_adjacency(n, &J.d_off, J.d_adj, true, s, &J.d_perm, nullptr);
        if (st != SLS_OK) return cleanup(st);
        e = launch_permute_coords(J.d_xy[0], J.d_xy[1], 0, false, n, J.d_perm, device_sm_count() * 4, s);
        std::swap(J.d_xy[0], J.d_xy[1]);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(J.d_xy[1], J.d_xy[0], cbytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(J.d_stats, 0, sizeof(PassStats) * (size_t)std::max(1, J.max_iter), s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&J.uploaded, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(J.uploaded, s);
    if (e != cudaSuccess) return cuda_err(e, "build");
    *footprint = built_footprint(n, da.adj_words, J.max_iter);
    return SLS_OK;
}

// Builds admitted jobs on the device, one at a time, on this thread's stream.
void builder_loop(sls_server *S, cudaStream_t s)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::shared_ptr<ServerJob> J;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_build.wait(lk, [S] { return S->stop || !S->to_build.empty(); });
            if (S->stop) break;
            J = S->to_build.front();
            S->to_build.pop_front();
        }
        size_t fp = 0;
        J->build_stream = s;
        const sls_status st = build_job(*J, groups_nodes(S->opt, J->n), s, &fp);
        const std::string err = st == SLS_OK ? std::string() : std::string(sls_last_error());
        if (st != SLS_OK) cudaStreamSynchronize(s);  // a failed build may leave an upload in flight
        J->release_inputs();  // once its uploads are done; outside the lock
        std::lock_guard<std::mutex> lk(S->mu);
        S->holding -= 1;
        if (st == SLS_OK) {
            S->used = S->used - J->reserved + fp;  // the scratch and the bound's slack return
            J->reserved = fp;
            J->upload_state = 1;
        } else {
            S->used -= J->reserved;
            J->reserved = 0;
            J->upload_state = 2;
            J->status = st;
            J->error = err;
        }
        S->cv_sched.notify_all();
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->builders_live -= 1;
    S->cv_sched.notify_all();
}

template <class T>
bool grow_host(T *&h, size_t &cap, size_t need)
{
    if (need <= cap) return true;
    const size_t c = std::max<size_t>(need, 2 * cap);
    cudaFreeHost(h);
    h = nullptr;
    cap = 0;
    if (cudaMallocHost((void **)&h, sizeof(T) * c) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cap = c;
    return true;
}

// cudaFree waits for the device, so a round in flight finishes before its
// buffers are replaced.
template <class T>
bool grow_dev(T *&d, size_t &cap, size_t need)
{
    if (need <= cap) return true;
    const size_t c = std::max<size_t>(need, 2 * cap);
    cudaFree(d);
    d = nullptr;
    cap = 0;
    if (cudaMalloc((void **)&d, sizeof(T) * c) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cap = c;
    return true;
}

// Rebuilds the job table and the warp-task list of the active set for the
// round launched next, whose parity is `slot`: the table and each job's
// first task are staged on the host, the task list is expanded on the device.
bool rebuild_table(sls_server *S, int slot)
{
    const size_t na = S->active.size();
    if (!grow_host(S->h_jobs[slot], S->jobs_hcap[slot], na) || !grow_dev(S->d_jobs, S->jobs_cap, na) ||
        !grow_host(S->h_toff[slot], S->toff_hcap[slot], na + 1) || !grow_dev(S->d_toff, S->toff_cap, na + 1))
        return false;
    JobDesc *hj = S->h_jobs[slot];
    int64_t *ht = S->h_toff[slot];
    int64_t t = 0;
    for (size_t j = 0; j < na; ++j) {
        ServerJob &J = *S->active[j];
        JobDesc &D = hj[j];
        D.xy[0] = J.d_xy[0];
        D.xy[1] = J.d_xy[1];
        D.node_off = J.d_off;
        D.adj = J.d_adj;
        D.n = J.n;
        D.stats = J.d_stats;
        const double thr = tolerance_threshold(J.tol, J.diag);
        std::memcpy(&D.thr_bits, &thr, sizeof thr);
        D.strict = S->opt.accept_strict;
        D.tol_active = J.tol > 0.0 ? 1 : 0;
        D.max_iter = J.max_iter;
        D.base_round = J.base_round;
        D.cur0 = 0;
        D.pad = 0;
        D.accept = nullptr;
        ht[j] = t;
        t += (J.n + 31) / 32;
    }
    ht[na] = t;
    if (!grow_dev(S->d_tasks, S->tasks_cap, (size_t)std::max<int64_t>(1, t))) return false;
    S->ntasks = t;
    return cudaMemcpyAsync(S->d_jobs, hj, sizeof(JobDesc) * na, cudaMemcpyHostToDevice, S->stream) == cudaSuccess &&
           cudaMemcpyAsync(S->d_toff, ht, sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, S->stream) ==
               cudaSuccess &&
           launch_expand_tasks(S->d_jobs, S->d_toff, (int)na, S->d_tasks, S->stream) == cudaSuccess;
}

// Copies the results of finished jobs to the host and frees their device
// memory, off the scheduler's thread: the next round starts at once.
void retire_loop(sls_server *S)
{
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<std::shared_ptr<ServerJob>> batch;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_retire.wait(lk, [S] { return S->retire_stop || !S->to_retire.empty(); });
            if (S->to_retire.empty()) return;  // stopping, and nothing left to retire
            batch.assign(S->to_retire.begin(), S->to_retire.end());
            S->to_retire.clear();
        }
        bool ok = true;
        // the round launched after a job's last one still reads its records:
        // wait for it before copying and freeing
        std::vector<cudaEvent_t> evs;
        for (auto &Jp : batch)
            if (Jp->free_after && std::find(evs.begin(), evs.end(), Jp->free_after) == evs.end())
                evs.push_back(Jp->free_after);
        for (cudaEvent_t ev : evs) ok = ok && cudaStreamWaitEvent(S->retire_stream, ev, 0) == cudaSuccess;
        for (auto &Jp : batch) {
            ServerJob &J = *Jp;
            const size_t rbytes = sizeof(double) * 2 * (size_t)J.n;
            if (J.result.cap < rbytes) {
                J.cache->put(J.result);
                try {
                    J.result = J.cache->get(rbytes);
                } catch (const std::bad_alloc &) {
                    ok = false;
                    continue;
                }
            }
            const double *res = J.d_xy[J.iterations & 1];
            if (J.d_perm) {
                // back to the caller's numbering, through the idle array
                double *d = J.d_xy[(J.iterations & 1) ^ 1];
                ok = ok && launch_unpermute_to_aos(res, 0, false, J.n, J.d_perm, d, device_sm_count() * 4,
                                                   S->retire_stream) == cudaSuccess;
                res = d;
            }
            ok = ok && cudaMemcpyAsync(J.result.p, res, rbytes, cudaMemcpyDeviceToHost, S->retire_stream) ==
                           cudaSuccess;
        }
        ok = ok && cudaStreamSynchronize(S->retire_stream) == cudaSuccess;  // one wait for the batch
        if (!ok) cudaGetLastError();
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
        for (auto &Jp : batch) Jp->free_after = nullptr;
        std::lock_guard<std::mutex> lk(S->mu);
        const auto now = Clock::now();
        for (auto &Jp : batch) {
            ServerJob &J = *Jp;
            free_job_device(J, S->retire_stream);
            S->used -= J.reserved;
            J.reserved = 0;
            if (ok) {
                J.t_done = now;
                J.state = kDone;
                S->latency_ms.push_back(std::chrono::duration<double, std::milli>(J.t_done - J.t_submit).count());
                S->node_updates += (double)J.n * (double)J.iterations;
                S->completed += 1;
            } else {
                fail_job(S, J, SLS_ERR_CUDA, "copying the result to the host failed");
            }
        }
        S->cv_done.notify_all();
        S->cv_sched.notify_all();
    }
}

// Whether the first queued job may be admitted: its bound fits the budget,
// or nothing else holds any (a job larger than its bound allows still gets
// its chance alone; its own allocations decide).
bool can_admit(const sls_server *S)
{
    if (S->queued.empty()) return false;
    const size_t need = S->queued.front()->reserved;
    return S->used + need <= S->budget || S->used == 0;
}

// Processes the records of a completed round over `jobs` (the active set it
// ran over): counts every job's executed pass and hands the jobs that reached
// their cap or tolerance to the retire thread.  Jobs already handed over in
// an earlier round are skipped (the round launched after their last pass
// still lists them, and skips them).  Returns the jobs that finished.
std::vector<std::shared_ptr<ServerJob>> process_round(sls_server *S, const std::vector<std::shared_ptr<ServerJob>> &jobs,
                                                      const PassStats *rec)
{
    std::vector<std::shared_ptr<ServerJob>> finished;
    for (size_t j = 0; j < jobs.size(); ++j) {
        ServerJob &J = *jobs[j];
        if (J.finished) continue;
        const PassStats &r = rec[j];
        bool done = true;  // a job with max_iter == 0 runs no pass
        if (J.max_iter > 0 && r.executed) {
            J.iterations += 1;
            J.info.iterations = J.iterations;
            J.info.accepted_last = (int64_t)r.nacc;
            std::memcpy(&J.info.max_d2_last, &r.maxd2_bits, sizeof(double));
            J.info.fp64_fallbacks += (int64_t)r.fallbacks;
            const double thr = tolerance_threshold(J.tol, J.diag);
            unsigned long long tb;
            std::memcpy(&tb, &thr, sizeof tb);
            const bool conv = J.tol > 0.0 && r.maxd2_bits < tb;
            J.info.converged = conv ? 1 : 0;
            done = conv || J.iterations >= J.max_iter;
        }
        if (done) {
            J.finished = true;
            finished.push_back(jobs[j]);
        }
    }
    return finished;
}

void scheduler_loop(sls_server *S)
{
    cudaSetDevice(S->device);
    bool dirty = true;
    // The round in flight (launched, records not yet read): its parity and
    // the active set it runs over.  Round r+1 is launched before the records
    // of round r are read, so the GPU never waits for the host between
    // rounds; a job that finished in round r is still listed in round r+1,
    // whose kernel skips it (its pass count or tolerance is reached).
    int pending = -1;
    std::vector<std::shared_ptr<ServerJob>> ran[2];
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_sched.wait(lk, [S, pending] {
                if (S->stop || !S->active.empty() || pending >= 0) return true;
                for (auto &J : S->uploading)
                    if (J->upload_state != 0) return true;
                return can_admit(S);
            });
            if (S->stop) break;
            bool handed = false;
            while (can_admit(S)) {
                auto J = S->queued.front();
                S->queued.pop_front();
                S->used += J->reserved;
                J->state = kBuilding;
                J->upload_state = 0;
                S->uploading.push_back(J);
                S->to_build.push_back(J);
                handed = true;
            }
            if (handed) S->cv_build.notify_all();
        }
        // built jobs join from the next round on (their builds overlap the
        // running rounds); with nothing running, wait for the first built one
        for (size_t k = 0; k < S->uploading.size();) {
            auto J = S->uploading[k];
            int ust;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                ust = J->upload_state;
                if (ust == 2) fail_job(S, *J, J->status, J->error);  // the builder freed its memory
            }
            if (ust == 2) {
                S->uploading.erase(S->uploading.begin() + k);
                continue;
            }
            if (ust == 0) {
                ++k;
                continue;
            }
            if (S->active.empty() && pending < 0) cudaEventSynchronize(J->uploaded);
            if (cudaEventQuery(J->uploaded) != cudaSuccess) {
                ++k;
                continue;
            }
            {
                std::lock_guard<std::mutex> lk(S->mu);
                J->base_round = S->round;
                J->state = kActive;
            }
            S->active.push_back(J);
            S->uploading.erase(S->uploading.begin() + k);
            dirty = true;
        }
        // launch the next round over the active set
        int launched = -1;
        if (!S->active.empty()) {
            const int slot = S->round & 1;
            const size_t na = S->active.size();
            if (dirty) {
                if (!rebuild_table(S, slot)) {
                    S->sched_error = "job table upload failed";
                    break;
                }
                dirty = false;
            }
            if (!grow_host(S->h_round[slot], S->round_cap[slot], na) ||
                !grow_dev(S->d_round[slot], S->dround_cap[slot], na)) {
                S->sched_error = "out of pinned host memory";
                break;
            }
            cudaError_t e = cudaEventRecord(S->ev_start[slot], S->stream);
            if (e == cudaSuccess)
                e = launch_batch_pass(S->d_jobs, S->d_tasks, S->ntasks, S->round, S->opt.layout, S->block, S->grid,
                                      S->stream, kServerChunk, nullptr);
            // every job's record of this round, gathered by one kernel, read back by one copy
            if (e == cudaSuccess) e = launch_gather_round(S->d_jobs, (int)na, S->round, S->d_round[slot], S->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(S->h_round[slot], S->d_round[slot], sizeof(PassStats) * na,
                                    cudaMemcpyDeviceToHost, S->stream);
            if (e == cudaSuccess) e = cudaEventRecord(S->ev_done[slot], S->stream);
            if (e != cudaSuccess) {
                S->sched_error = cudaGetErrorString(e);
                cudaGetLastError();
                break;
            }
            ran[slot] = S->active;
            S->round += 1;
            launched = slot;
        }
        // read the round launched before this one
        if (pending >= 0) {
            cudaError_t e = cudaEventSynchronize(S->ev_done[pending]);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, S->ev_start[pending], S->ev_done[pending]);
            if (e != cudaSuccess) {
                S->sched_error = cudaGetErrorString(e);
                cudaGetLastError();
                break;
            }
            S->busy_s += 1e-3 * (double)ms;
            auto finished = process_round(S, ran[pending], S->h_round[pending]);
            ran[pending].clear();
            if (!finished.empty()) {
                // their memory is released once the round just launched (which
                // still reads their records) is done
                cudaEvent_t ev = nullptr;
                if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventRecord(ev, S->stream) != cudaSuccess) {
                    S->sched_error = "event for finished jobs";
                    cudaGetLastError();
                    break;
                }
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    for (auto &Jp : finished) {
                        Jp->state = kRetiring;
                        Jp->free_after = ev;
                        S->to_retire.push_back(Jp);
                    }
                }
                S->cv_retire.notify_one();
                std::vector<std::shared_ptr<ServerJob>> keep;
                keep.reserve(S->active.size());
                for (auto &Jp : S->active)
                    if (!Jp->finished) keep.push_back(Jp);
                S->active.swap(keep);
                dirty = true;
            }
        }
        pending = launched;
    }
    // cancel what is left, once no builder touches a job any more
    std::unique_lock<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_build.notify_all();
    S->cv_sched.wait(lk, [S] { return S->builders_live == 0; });
    for (auto &J : S->active) {
        free_job_device(*J, S->stream);
        S->used -= J->reserved;
        fail_job(S, *J, SLS_ERR_NOT_FOUND, "server destroyed before the job finished");
    }
    S->active.clear();
    for (auto &J : S->uploading) {
        // built or failed by a builder (memory on its stream), or never started
        if (J->upload_state == 1) free_job_device(*J, J->build_stream);
        if (J->upload_state != 2) S->used -= J->reserved;
        fail_job(S, *J, SLS_ERR_NOT_FOUND, "server destroyed before the job finished");
    }
    S->uploading.clear();
    S->to_build.clear();
    for (auto &J : S->queued) fail_job(S, *J, SLS_ERR_NOT_FOUND, "server destroyed before the job started");
    S->queued.clear();
    if (!S->sched_error.empty())
        for (auto &kv : S->jobs)
            if (kv.second->state != kDone && kv.second->state != kFailed && kv.second->state != kRetiring)
                fail_job(S, *kv.second, SLS_ERR_CUDA, "scheduler stopped on a CUDA error");
    lk.unlock();
    cudaStreamSynchronize(S->stream);
}

}  // namespace

extern "C" {

sls_status sls_server_create(size_t hbm_budget, int32_t max_queue, const sls_options *opt, sls_server **out)
{
    if (!out) return fail(SLS_ERR_INVALID, "out must not be NULL");
    *out = nullptr;
    if (max_queue < 0) return fail(SLS_ERR_INVALID, "max_queue must be >= 0");
    sls_options o = resolve_options(opt);
    sls_status st = check_options(o);
    if (st != SLS_OK) return st;
    if (o.form != 0 || o.precision != 64) return fail(SLS_ERR_INVALID, "the server runs FP64 Form A only");
    if (o.skip_unchanged) return fail(SLS_ERR_INVALID, "the server computes every tile (skip_unchanged is for single meshes)");
    if (o.layout != 0) return fail(SLS_ERR_INVALID, "the server keeps coordinates interleaved (layout = 0)");
    auto S = std::make_unique<sls_server>();
    S->opt = o;
    S->max_queue = max_queue;
    if (cudaGetDevice(&S->device) != cudaSuccess) return fail(SLS_ERR_CUDA, "cudaGetDevice failed");
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return fail(SLS_ERR_CUDA, "cudaMemGetInfo failed");
    S->budget = hbm_budget ? hbm_budget : (size_t)(0.8 * (double)free_b);
    // builders: each uploads and builds one job at a time on its own stream
    const int nb = std::min(kBuilders, std::max(1, (int)std::thread::hardware_concurrency()));
    S->build_streams.assign(nb, nullptr);
    bool streams_ok = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&S->retire_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &bs : S->build_streams)
        streams_ok = streams_ok && cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2; ++b)
        streams_ok = streams_ok && cudaEventCreate(&S->ev_start[b]) == cudaSuccess &&
                     cudaEventCreate(&S->ev_done[b]) == cudaSuccess;
    if (!streams_ok) {
        cudaGetLastError();
        for (int b = 0; b < 2; ++b) {
            if (S->ev_start[b]) cudaEventDestroy(S->ev_start[b]);
            if (S->ev_done[b]) cudaEventDestroy(S->ev_done[b]);
        }
        for (cudaStream_t x : S->build_streams)
            if (x) cudaStreamDestroy(x);
        if (S->stream) cudaStreamDestroy(S->stream);
        if (S->retire_stream) cudaStreamDestroy(S->retire_stream);
        return fail(SLS_ERR_CUDA, "stream or event creation failed");
    }
    S->block = (opt != nullptr && opt->block_size >= 32 && opt->block_size <= 128) ? opt->block_size : 128;
    S->grid = device_sm_count() * batch_pass_occupancy(o.layout, S->block);
    sls_server *raw = S.release();
    raw->builders_live = nb;
    for (int b = 0; b < nb; ++b) raw->builders.emplace_back(builder_loop, raw, raw->build_streams[b]);
    raw->retirer = std::thread(retire_loop, raw);
    raw->sched = std::thread(scheduler_loop, raw);
    *out = raw;
    return SLS_OK;
}

sls_status sls_submit(sls_server *S, const double *xy, int64_t n, const int32_t *tri, int64_t m,
                      const uint8_t *boundary, int32_t max_iter, double tol_rel, uint64_t *job)
{
    if (!S || !xy || !tri || !job) return fail(SLS_ERR_INVALID, "server, xy, tri and job must not be NULL");
    if (n < 3 || m < 1 || n >= (int64_t(1) << 31) || m >= (int64_t(1) << 31))
        return fail(SLS_ERR_INVALID, "bad mesh size");
    if (max_iter < 0 || std::isnan(tol_rel)) return fail(SLS_ERR_INVALID, "bad stop rule");
    // what the job holds at least once built: coordinates and offsets alone
    const size_t least = 2 * sizeof(double) * 2 * (size_t)n + sizeof(uint32_t) * (size_t)(n + 1);
    if (least > S->budget) return fail(SLS_ERR_REJECTED, "job larger than the server's memory budget");
    const auto t_submit = Clock::now();
    {
        // take the queue place first, so that a full queue costs no copy
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->max_queue > 0 && S->holding >= S->max_queue)
            return fail(SLS_ERR_BUSY, "server queue is full");
        S->holding += 1;
    }
    std::shared_ptr<ServerJob> J;
    try {
        // copy the inputs outside the server's lock, which every thread needs
        J = std::make_shared<ServerJob>();
        J->cache = S->pinned;
        const size_t bx = sizeof(double) * 2 * (size_t)n, bt = sizeof(int32_t) * 3 * (size_t)m;
        J->in = S->pinned->get(bx + bt + (boundary ? (size_t)n : 0));
        char *base = static_cast<char *>(J->in.p);
        std::memcpy(base, xy, bx);
        std::memcpy(base + bx, tri, bt);
        J->xy = reinterpret_cast<const double *>(base);
        J->tri = reinterpret_cast<const int32_t *>(base + bx);
        if (boundary) {
            std::memcpy(base + bx + bt, boundary, (size_t)n);
            J->boundary = reinterpret_cast<const uint8_t *>(base + bx + bt);
        }
    } catch (const std::bad_alloc &) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->holding -= 1;
        return fail(SLS_ERR_OOM, "host allocation failed");
    }
    J->t_submit = t_submit;
    J->n = n;
    J->m = m;
    J->max_iter = max_iter;
    J->tol = tol_rel;
    J->reserved = admission_bound(n, m, max_iter);
    std::lock_guard<std::mutex> lk(S->mu);
    J->id = S->next_id++;
    S->jobs[J->id] = J;
    S->queued.push_back(J);
    S->cv_sched.notify_all();
    *job = J->id;
    return SLS_OK;
}

sls_status sls_wait(sls_server *S, uint64_t job, double timeout_s, double *xy_out, sls_info *info)
{
    if (!S) return fail(SLS_ERR_INVALID, "server must not be NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(job);
    if (it == S->jobs.end()) return fail(SLS_ERR_NOT_FOUND, "unknown job id");
    std::shared_ptr<ServerJob> J = it->second;
    auto ready = [&J] { return J->state == kDone || J->state == kFailed; };
    if (timeout_s < 0.0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return fail(SLS_ERR_TIMEOUT, "job not finished within the timeout");
    }
    // an oversized job is only known after its adjacency is built
    S->jobs.erase(job);
    if (J->state == kFailed) return fail(J->status, J->error);
    // the copy of a large result must not hold up the scheduler and the
    // builders: the job is ours alone once it left the table
    lk.unlock();
    if (xy_out) std::memcpy(xy_out, J->result.p, sizeof(double) * 2 * (size_t)J->n);
    if (info) *info = J->info;
    return SLS_OK;
}

sls_status sls_server_stats(const sls_server *Sc, double *p50_ms, double *p99_ms, double *nups, int64_t *completed)
{
    if (!Sc) return fail(SLS_ERR_INVALID, "server must not be NULL");
    sls_server *S = const_cast<sls_server *>(Sc);
    std::lock_guard<std::mutex> lk(S->mu);
    std::vector<double> v = S->latency_ms;
    auto pct = [&v](double p) {
        if (v.empty()) return 0.0;
        const size_t k = std::min(v.size() - 1, (size_t)std::ceil(p / 100.0 * (double)v.size()) - (p > 0 ? 1 : 0));
        std::nth_element(v.begin(), v.begin() + k, v.end());
        return v[k];
    };
    if (p50_ms) *p50_ms = pct(50.0);
    if (p99_ms) *p99_ms = pct(99.0);
    if (nups) *nups = S->busy_s > 0.0 ? S->node_updates / S->busy_s : 0.0;
    if (completed) *completed = S->completed;
    return SLS_OK;
}

sls_status sls_server_destroy(sls_server *S)
{
    if (!S) return SLS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_build.notify_all();
    S->cv_sched.notify_all();
    // the scheduler cancels what is left once every builder has stopped
    if (S->sched.joinable()) S->sched.join();
    for (auto &t : S->builders) t.join();
    {
        // the scheduler has stopped handing over jobs: finish what it handed over
        std::lock_guard<std::mutex> lk(S->mu);
        S->retire_stop = true;
    }
    S->cv_retire.notify_all();
    if (S->retirer.joinable()) S->retirer.join();
    for (cudaStream_t bs : S->build_streams) cudaStreamSynchronize(bs);
    cudaStreamSynchronize(S->retire_stream);
    cudaStreamSynchronize(S->stream);
    for (int b = 0; b < 2; ++b) {
        cudaFreeHost(S->h_jobs[b]);
        cudaFreeHost(S->h_toff[b]);
        cudaFreeHost(S->h_round[b]);
        cudaFree(S->d_round[b]);
        if (S->ev_start[b]) cudaEventDestroy(S->ev_start[b]);
        if (S->ev_done[b]) cudaEventDestroy(S->ev_done[b]);
    }
    cudaFree(S->d_jobs);
    cudaFree(S->d_toff);
    cudaFree(S->d_tasks);
    cudaStreamDestroy(S->stream);
    cudaStreamDestroy(S->retire_stream);
    for (cudaStream_t bs : S->build_streams) cudaStreamDestroy(bs);
    delete S;
    return SLS_OK;
}

}  // extern "C"
