/*
 * slsmooth.h -- C ABI of the GB300 (sm_103a) library for two-dimensional
 * Smart Laplacian mesh smoothing (Zhao, Mei, Xu, Zhang, "On the Accelerating
 * of Two-dimensional Smart Laplacian Smoothing on the GPU").
 *
 * What the library computes (the paper's method, Form A):
 *   - every free node moves to the centre of its neighbours (Eq. 2), computed
 *     from the coordinates of the previous pass only (Jacobi);
 *   - the move is kept only if the worst quality of the node's incident
 *     triangles does not get worse (Section 2.1, Section 3.3.4); quality is
 *     Lee and Lo's alpha (Section 3.3.1);
 *   - boundary nodes are fixed (Section 3.3.3).
 *
 * Fixed readings where the paper is silent (the test suite's CPU oracle uses
 * the same ones):
 *   - neighbours are summed in ascending (x0, y0, index) order, (x0, y0) being
 *     the coordinates passed to sls_mesh_create;
 *   - alpha = 2*sqrt(3) * cross / (|e1|^2 + |e2|^2 + |e3|^2) with e1 = b-a,
 *     e2 = c-a, e3 = c-b of the triangle (a, b, c) in its stored vertex order,
 *     cross = e1x*e2y - e1y*e2x (signed: inverted triangles score below 0),
 *     the sum taken as (|e1|^2 + |e2|^2) + |e3|^2, and alpha = 0 if the sum is
 *     not positive;
 *   - accept iff q_new >= q_old (accept_strict = 1: q_new > q_old);
 *   - the squared move of an accepted node is dx*dx + dy*dy with dx = cx - x;
 *   - with tol_rel > 0 a run stops after the first pass whose largest squared
 *     move is below (tol_rel * D)^2, D being the bounding-box diagonal of the
 *     coordinates passed to sls_mesh_create.
 * All arithmetic is IEEE-754 binary64 with round-to-nearest and no
 * contraction, so results are bit-identical to a sequential CPU evaluation of
 * the same expressions.
 *
 * Conventions
 *   - Every entry point returns an sls_status and never throws.  On failure
 *     sls_last_error() describes the problem (thread-local string).
 *   - Host buffers are owned by the caller and only read (or written) during
 *     the call.  The library owns all device memory it allocates.
 *   - A handle (sls_mesh, sls_batch, sls_server) is not thread-safe; distinct
 *     handles may be used from distinct threads.  sls_server is the exception:
 *     sls_submit / sls_wait may be called from any thread.
 *   - Coordinates are interleaved (x0, y0, x1, y1, ...) float64 on the host.
 *   - Limits: 3 <= n < 2^31 nodes, 1 <= m < 2^31 triangles, at most 32767
 *     neighbours per node, total adjacency words < 2^32.
 */
#ifndef SLSMOOTH_H
#define SLSMOOTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sls_status {
    SLS_OK = 0,
    SLS_ERR_INVALID = 1,     /* bad argument, bad index, repeated vertex, non-finite coordinate */
    SLS_ERR_NONMANIFOLD = 2, /* an edge shared by more than two triangles                        */
    SLS_ERR_OOM = 3,         /* device or host allocation failed / over the memory budget        */
    SLS_ERR_CUDA = 4,        /* a CUDA runtime call failed (message in sls_last_error)           */
    SLS_ERR_TIMEOUT = 5,     /* a bounded device-side or host-side wait ran out                  */
    SLS_ERR_BUSY = 6,        /* the server queue is full                                         */
    SLS_ERR_REJECTED = 7,    /* the job can never fit the server's memory budget                 */
    SLS_ERR_NOT_FOUND = 8    /* unknown job id                                                   */
} sls_status;

/* Kernel choice for the Jacobi pass. */
enum {
    SLS_KERNEL_AUTO = 0,      /* the fastest exact kernel                                  */
    SLS_KERNEL_FP64 = 1,      /* one thread per node, every step on the FP64 pipe          */
    SLS_KERNEL_FILTERED = 2   /* exact: FP32 screening of the accept test, FP64 where needed */
};

typedef struct sls_options {
    int32_t accept_strict; /* 0: accept iff q_new >= q_old (default); 1: q_new > q_old       */
    int32_t copy_back;     /* 0: ping-pong the two coordinate arrays (default);
                              1: copy the new pass back over the old one after every pass
                              (the paper's "swapping" of intermediate coordinates)          */
    int32_t layout;        /* 0: AoS, one double2 per node (default); 1: SoA, x[] then y[]   */
    int32_t kernel;        /* SLS_KERNEL_*                                                   */
    int32_t record_accept; /* 1: keep the per-node accept decisions of the last pass         */
    int32_t block_size;    /* threads per block; 0 = library default                         */
    int32_t l2_window;     /* 1: each pass marks the coordinates it gathers from as
                              persisting in L2 (a stream access-policy window; the share
                              that fits the context's persisting carve-out, which this
                              sets with cudaDeviceSetLimit), cleared when sls_smooth
                              returns.  Same results; see the measured effect before use.  */
    int32_t passes_per_check; /* passes launched between host checks of the stop rule; 0 = 16 */
    int32_t host_build;    /* 1: build the adjacency on the host; 0: on the device (default;
                              the host build is still used for nodes in more than 32
                              triangles)                                                     */
    int32_t form;          /* 0: Form A, the Jacobi pass of Eq. 2 (default).  1: Form B
                              (Eq. 3, in place) made deterministic as multicolour
                              Gauss-Seidel: the free nodes are coloured at creation so that
                              no two neighbours share a colour (Jones-Plassmann rounds,
                              priority splitmix64(150200355 + node id)), and every sweep
                              updates the colour classes in turn, in place.  Inside the
                              library the mesh is renumbered so that each class is a
                              contiguous id range (8 bytes per node for the maps); every
                              call still reads and writes coordinates and decisions in the
                              caller's numbering.  copy_back is ignored.  Single meshes
                              only: the batched, served, allocation-free and gather /
                              scatter entry points reject it.                                */
    int32_t precision;     /* 64 (default; 0 means 64): FP64 coordinates and arithmetic,
                              results bit-identical to the FP64 definition.  32: binary32
                              coordinates (the given doubles rounded to nearest) and every
                              operation one binary32 round-to-nearest operation in the same
                              order, the paper's precision (Section 4).  Single meshes only. */
    int32_t skip_unchanged;/* 1: from the second pass of an sls_smooth call on, a tile of 32
                              consecutive nodes is not recomputed when none of its nodes and
                              none of their neighbours changed coordinates in the previous
                              pass: its inputs are then those of the previous pass, so its
                              coordinates and decisions are too (Form A is a function of the
                              previous pass only, Eq. 2).  Results are identical to 0; the
                              gain grows as the mesh settles.  Needs form = 0, precision = 64
                              and the screened kernel (SLS_KERNEL_AUTO or _FILTERED); costs
                              140 bytes of device memory per 32 nodes.  The batched and
                              allocation-free forms compute every tile; the server rejects it. */
    int32_t numbering;     /* FP64: 0 (default) lets the library renumber a mesh of at least
                              2^20 nodes, 1 keeps the caller's numbering, 2 renumbers at any
                              size (binary32 meshes keep it: their pass gains nothing).
                              Form A: every window of 128 consecutive ids lists its nodes by
                              incident-triangle count, then degree (fixed nodes last, ties by
                              id); Form B: the same inside each colour class's range.  The 32
                              lanes of a warp then run loops of similar length (the pass's
                              loops run to the warp's longest).  The windows
                              stay where they are, so the gathers keep their locality.  Costs
                              two kernels and 8 bytes per node at creation, which only larger
                              meshes repay.  Not done with skip_unchanged (its 32-node tiles
                              would lose their locality).  Every call still reads and writes
                              coordinates, decisions and node ids in the caller's numbering;
                              results are identical.                                         */
    void *stream;          /* cudaStream_t to run on; NULL = a stream owned by the handle    */
} sls_options;

typedef struct sls_info {
    int32_t iterations;    /* passes executed by the last sls_smooth call                    */
    int32_t converged;     /* 1 if the tolerance stopped the run                              */
    int64_t accepted_last; /* accepted free nodes in the last executed pass                   */
    double max_d2_last;    /* largest squared move in the last executed pass                  */
    int64_t fp64_fallbacks;/* accept tests the screened kernel re-did in FP64 (last call)     */
    int64_t launches;      /* kernel launches issued by the last sls_smooth call (passes
                              launched after the tolerance was met return at once; 0 from
                              the batched and served forms)                                 */
    int64_t nodes_skipped; /* node updates not recomputed by the last sls_smooth call
                              (skip_unchanged: the nodes of the skipped tiles, summed over
                              its passes)                                                   */
} sls_info;

typedef struct sls_mesh sls_mesh;
typedef struct sls_batch sls_batch;
typedef struct sls_server sls_server;

/* Fills *opt with the defaults. */
void sls_default_options(sls_options *opt);

/* Builds a mesh handle: validates the input, finds every node's neighbours
 * and incident triangles (Section 3.3.2), determines the constraints
 * (Section 3.3.3: with boundary == NULL a node is fixed when one of its
 * edges belongs to a single triangle, or when it is in no triangle), and
 * uploads adjacency and coordinates to the current CUDA device.
 *   xy       host, 2n float64, interleaved
 *   tri      host, 3m int32 vertex ids; the vertex order of each triangle is
 *            kept and defines the sign of its quality
 *   boundary host, n uint8 (nonzero = fixed), or NULL to derive the flags
 *   opt      NULL for defaults; copied
 *   out      receives the handle (NULL on failure)
 * Errors: SLS_ERR_INVALID, SLS_ERR_NONMANIFOLD, SLS_ERR_OOM, SLS_ERR_CUDA. */
sls_status sls_mesh_create(const double *xy, int64_t n, const int32_t *tri, int64_t m,
                           const uint8_t *boundary, const sls_options *opt, sls_mesh **out);

/* Runs up to max_iter Jacobi passes of Smart Laplacian smoothing (Eq. 2 with
 * the accept test of Section 3.3.4), continuing from the handle's current
 * coordinates.  tol_rel <= 0 disables the tolerance stop.  info may be NULL.
 * Blocks until the passes are done. */
sls_status sls_smooth(sls_mesh *mesh, int32_t max_iter, double tol_rel, sls_info *info);

/* Copies the current coordinates (2n float64, interleaved) to xy_out, which is
 * host memory (dst_is_device = 0) or device memory of the mesh's device
 * (dst_is_device = 1, copied on the handle's stream and synchronised). */
sls_status sls_get_coords(const sls_mesh *mesh, double *xy_out, int32_t dst_is_device);

/* Overwrites the current coordinates (2n float64, interleaved), read from host
 * memory (src_is_device = 0) or from device memory of the mesh's device
 * (src_is_device = 1).  Adjacency, the summation order and D stay those of
 * sls_mesh_create.  Host input is checked to be finite; device input is not.
 * Device input is read on the handle's stream, so work on another stream that
 * writes it must be complete (or ordered before that stream) at the call; the
 * call returns once the coordinates are in place. */
sls_status sls_set_coords(sls_mesh *mesh, const double *xy, int32_t src_is_device);

/* Ghost exchange of a mesh split over several GPUs (a build addition: the
 * paper runs on one GPU).  Form A reads only the previous pass (Eq. 2), so a
 * mesh split into subdomains, each holding its nodes plus a one-ring of
 * ghost nodes (fixed in the subdomain's mesh), gives the same passes as the
 * whole mesh when every ghost gets its owner's coordinates between passes.
 *   sls_gather_coords  copies the current coordinates of the k nodes idx[]
 *                      (device int32, ids of this mesh) to out (device, 2k
 *                      float64 interleaved);
 *   sls_scatter_coords writes in (device, 2k float64) into both coordinate
 *                      arrays of the k listed nodes (distinct ids).
 * Ids are in the caller's numbering (mapped inside the library when it
 * renumbered the mesh).  Both run on the handle's stream and return when
 * done.  FP64 Form-A meshes only.
 * Errors: SLS_ERR_INVALID for an id outside [0, n) (nothing is written for
 * it), a binary32 or a Form-B mesh. */
sls_status sls_gather_coords(sls_mesh *mesh, const int32_t *idx, int64_t k, double *out);
sls_status sls_scatter_coords(sls_mesh *mesh, const int32_t *idx, int64_t k, const double *in);

/* Copies the accept decisions of the last executed pass (n uint8, host;
 * 1 = moved to the centre).  Needs opt->record_accept = 1. */
sls_status sls_get_accept(const sls_mesh *mesh, uint8_t *accept_out);

/* Quality histogram of all triangles at the current coordinates
 * (Section 3.3.1): bin = floor((q - lo) / (hi - lo) * nbins) clamped to
 * [0, nbins-1]; counts (host, nbins int64), qmin, qmean (either may be NULL).
 * qmean is summed in an order of the library's choosing. */
sls_status sls_quality_histogram(const sls_mesh *mesh, int32_t nbins, double lo, double hi,
                                 int64_t *counts, double *qmin, double *qmean);

/* Node and triangle counts, free nodes and D. */
sls_status sls_mesh_stats(const sls_mesh *mesh, int64_t *n, int64_t *m, int64_t *n_free,
                          double *diag);

/* Frees the handle.  Its device memory goes back to the library's memory
 * pool on the device (see sls_trim_memory); returns without waiting for the
 * device. */
sls_status sls_mesh_destroy(sls_mesh *mesh);

/* Device memory of meshes, their builds and served jobs comes from one
 * stream-ordered memory pool per device that the library owns (the device's
 * default pool is left alone).  Memory that destroyed handles return stays
 * in the pool for later handles, so creating a mesh of a size seen before
 * maps no new memory.  sls_trim_memory waits for the current device and then
 * hands the pool's unused memory back to the driver, keeping at most
 * keep_bytes.  Not a counterpart of anything in the paper: a memory policy of
 * this library. */
sls_status sls_trim_memory(size_t keep_bytes);

/* ---- batched form: many meshes of uneven size, one graph launch --------
 * Each mesh keeps its own device buffers, iteration count and tolerance; the
 * batch adds a job table and a list of 32-node work items, and runs round r
 * (pass r of every mesh with passes left) as one kernel launch; all rounds of
 * a call are replayed from one CUDA graph.  Results are bit-identical to
 * smoothing each mesh alone with sls_smooth. */

/* Packs k distinct mesh handles (same device, same layout) into one batch.
 * iters (k int32) and tol_rel (k float64, may be NULL = off) are the per-mesh
 * stop rules.  The handles must outlive the batch; sls_batch_smooth advances
 * their coordinates in place.  The coordinates at packing time are saved for
 * sls_batch_reset.  The launch shape is autotuned by timing one full batch
 * smooth per candidate, restoring the saved coordinates after each trial:
 * the chunk of consecutive 32-node tasks a warp takes (one contiguous share
 * of the list per warp, 64 in a grid stride, or 32 claimed in order from a
 * per-round counter) and, with opt == NULL or
 * opt->block_size == 0, the block size (64 or 128 threads); an explicit
 * block_size must be 32, 64, 96 or 128 (SLS_ERR_INVALID otherwise). */
sls_status sls_batch_create(sls_mesh *const *meshes, int32_t k, const int32_t *iters,
                            const double *tol_rel, const sls_options *opt, sls_batch **out);

/* Smooths every mesh of the batch to its own stop rule (continuing from each
 * mesh's current coordinates).  infos (k, may be NULL) receives the per-mesh
 * results in packing order. */
sls_status sls_batch_smooth(sls_batch *batch, sls_info *infos);

/* Coordinates of mesh j of the batch (host, 2 n_j float64). */
sls_status sls_batch_get_coords(const sls_batch *batch, int32_t j, double *xy_out);

/* Restores every mesh of the batch to the coordinates it had when packed. */
sls_status sls_batch_reset(sls_batch *batch);

/* The launch shape in use (chosen by the autotuner, or set below): threads
 * per block and the warp chunk (> 0: tasks per chunk in a grid stride; < 0:
 * chunks of -chunk tasks claimed in order from a per-round counter; 0: one
 * contiguous share of the task list per warp).  Either pointer may be NULL. */
sls_status sls_batch_shape(const sls_batch *batch, int32_t *block, int64_t *chunk);

/* Sets the launch shape (block 32, 64, 96 or 128; |chunk| <= 2^20) for the
 * following sls_batch_smooth calls, e.g. to repeat a tuned shape without
 * tuning again.  Results do not depend on the shape. */
sls_status sls_batch_set_shape(sls_batch *batch, int32_t block, int64_t chunk);

sls_status sls_batch_destroy(sls_batch *batch);

/* ---- served form: jobs arrive over time (continuous batching) -----------
 * A scheduler thread admits queued jobs in arrival order while a bound on
 * their device footprint (coordinates, adjacency, statistics and the
 * adjacency build's scratch, about 70n + 84m bytes) fits the memory budget;
 * a job is also admitted when the server holds nothing else.  Builder
 * threads, each with its own stream, upload admitted jobs and build their
 * adjacency on the device (stream-ordered allocations from the library's
 * memory pool, so the running rounds are never synchronised; a mesh
 * with a node in more than 32 triangles is built on the host).  The
 * scheduler runs every built job's next pass in one launch per round and
 * retires each job at its own iteration cap or tolerance. */

/* hbm_budget: bytes of device memory the server may hold for jobs (0 = 80%
 * of the free memory at creation).  max_queue: jobs submitted but not yet
 * built on the device (the jobs whose inputs the server still holds in host
 * memory) that sls_submit accepts (0 = unlimited); beyond it sls_submit
 * returns SLS_ERR_BUSY.  opt: FP64 Form A with the AoS layout only
 * (SLS_ERR_INVALID otherwise).  opt's numbering applies to every job as to
 * a single mesh (by default jobs of 2^20 nodes or more are renumbered;
 * results in the caller's numbering; 4 bytes per node more while held).
 * Jobs take their device memory from the library's
 * pool (see sls_trim_memory); their inputs and results wait in page-locked
 * host memory, of which the server keeps up to 4 GiB for reuse until it is
 * destroyed. */
sls_status sls_server_create(size_t hbm_budget, int32_t max_queue, const sls_options *opt,
                             sls_server **out);

/* Queues one smoothing job; inputs are copied before returning.  *job
 * receives its id.  Errors: SLS_ERR_INVALID (bad sizes or stop rule),
 * SLS_ERR_REJECTED (its coordinates and offsets alone exceed the budget),
 * SLS_ERR_BUSY (queue full).  A mesh that fails validation (bad index,
 * repeated vertex, non-finite coordinate, non-manifold edge) is reported by
 * sls_wait with the same status sls_mesh_create would return. */
sls_status sls_submit(sls_server *srv, const double *xy, int64_t n, const int32_t *tri, int64_t m,
                      const uint8_t *boundary, int32_t max_iter, double tol_rel, uint64_t *job);

/* Waits up to timeout_s seconds (< 0: forever) for a job; copies its final
 * coordinates (host, 2n float64; may be NULL) and info, then forgets the job.
 * SLS_ERR_TIMEOUT if it is not done in time (the job stays). */
sls_status sls_wait(sls_server *srv, uint64_t job, double timeout_s, double *xy_out,
                    sls_info *info);

/* Latency percentiles (submit to result ready on the host, milliseconds) of
 * the jobs completed so far, and node-updates per second over the busy time. */
sls_status sls_server_stats(const sls_server *srv, double *p50_ms, double *p99_ms,
                            double *node_updates_per_s, int64_t *completed);

sls_status sls_server_destroy(sls_server *srv);

/* ---- smoothing without allocation ---------------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory when they smooth: latency-critical loops that
 * must not pay the device-wide synchronisation of cudaMalloc/cudaFree,
 * plug-ins whose host application has reserved all device memory for its own
 * pool (a framework's caching allocator, for one), and services that fix
 * their memory budget at start-up and must not fail for lack of memory later.
 *
 * Runs the same passes as sls_smooth on the mesh's adjacency, but on two
 * coordinate buffers the caller owns, and calls no cudaMalloc, cudaFree or
 * other allocating routine.  The only scratch the kernels need -- one
 * 32-byte statistics record per pass -- lives in a fixed array of
 * SLS_NOALLOC_MAX_PASSES records (128 KiB) in device global memory, part of
 * the library image.  CUDA loads a library's device code and data lazily;
 * sls_mesh_create (which allocates anyway) loads this array on the mesh's
 * device, so this call finds it in place and loads nothing itself.  Every GPU
 * on which a mesh was created holds the array until the process exits.
 *   mesh     a handle created with the AoS layout (layout = 0), Form A and
 *            FP64; its own coordinates, accept mask and statistics are not
 *            used or changed, and its copy_back, skip_unchanged, l2_window and
 *            record_accept options are not applied (the results are the
 *            same: those options never change them).  When the library
 *            renumbered the mesh (see numbering) two more kernels map
 *            the coordinates into its numbering and back; both buffers are
 *            in the caller's numbering
 *   xy_in    device, 2n float64 interleaved: the starting coordinates; also
 *            serves as the second buffer of the ping-pong, so its contents
 *            are unspecified on return
 *   xy_out   device, 2n float64: receives the result (distinct from xy_in)
 *   max_iter 0 .. SLS_NOALLOC_MAX_PASSES; larger values are rejected with
 *            SLS_ERR_INVALID
 *   stream   cudaStream_t, or NULL for the mesh's stream; the call returns
 *            after the work on it is done
 * Results are bit-identical to sls_smooth on the same coordinates.  The
 * mesh's device must be current.  The array's device address is looked up
 * by sls_mesh_create and again after the device's context changes (after
 * cudaDeviceReset); the lookup neither loads nor allocates once the array is
 * in place.  The array is cleared at the start of each call and keeps the
 * last call's records afterwards.  All calls on a device
 * share it: calls whose work overlaps on the GPU (other threads, other
 * streams) race and must be serialised by the caller. */
#define SLS_NOALLOC_MAX_PASSES 4096
sls_status sls_smooth_noalloc(const sls_mesh *mesh, double *xy_in, double *xy_out, int32_t max_iter,
                              double tol_rel, void *stream, sls_info *info);

const char *sls_status_str(sls_status s);
const char *sls_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SLSMOOTH_H */
