// kernels.h -- host-callable launchers of the slsmooth CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "device.cuh"

namespace sls {

// One Jacobi pass, every step on the FP64 pipe (one thread per node).
cudaError_t launch_pass_fp64(const PassArgs &a, int layout, int block, int grid, cudaStream_t s);
// Blocks per SM the FP64 pass kernel can keep resident at `block` threads.
int pass_fp64_occupancy(int layout, int block);

// One Jacobi pass, screened: FP64 neighbour sums in the stored order, the
// division by the degree as one FP64 multiplication plus an exact integer
// correction, FP32 screening of the accept test, FP64 quality only where the
// screen cannot decide (bit-identical results).
cudaError_t launch_pass_screened(const PassArgs &a, int layout, int block, int grid, cudaStream_t s);
int pass_screened_occupancy(int layout, int block);

// One round of the batched / served form over all active jobs' tasks.
// chunk > 0: tasks per warp chunk, taken in a grid stride; chunk < 0: chunks
// of -chunk tasks claimed in order from *claim (zero at the launch); 0 = one
// contiguous share of the task list per warp.
cudaError_t launch_batch_pass(const JobDesc *jobs, const WarpTask *tasks, int64_t ntasks, int round,
                              int layout, int block, int grid, cudaStream_t s, int64_t chunk,
                              unsigned long long *claim);
int batch_pass_occupancy(int layout, int block);
// The warp tasks of the na jobs of a table (job j's tasks from task_off[j]).
cudaError_t launch_expand_tasks(const JobDesc *jobs, const int64_t *task_off, int na, WarpTask *tasks,
                                cudaStream_t s);
// Record of round `round` of each of the na jobs (pass round - base_round,
// clamped to the job's last pass) into out[0 .. na).
cudaError_t launch_gather_round(const JobDesc *jobs, int na, int round, PassStats *out, cudaStream_t s);

// Copy-back form: out -> in after pass q (skipped when pass q was skipped).
cudaError_t launch_copy_back(const double *src, double *dst, int64_t n_doubles,
                             const PassStats *stats, int q, int grid, cudaStream_t s);

// Quality histogram of all triangles (counts must be zeroed by the caller;
// qmin_key is the order-preserving key of the minimum, init 0xff..ff;
// qsum accumulates the qualities).
cudaError_t launch_histogram(const double *xy, int layout, int64_t n, const int32_t *tri,
                             int64_t m, int nbins, double lo, double hi,
                             unsigned long long *counts, unsigned long long *qmin_key,
                             double *qsum, int grid, cudaStream_t s);

// One pass in binary32 (pass_f32.cu): a.in / a.out hold floats.
cudaError_t launch_pass_f32(const PassArgs &a, int layout, int block, int grid, cudaStream_t s);
int pass_f32_occupancy(int layout, int block);
// Copy-back form of the binary32 pass (count floats; skipped when pass q was skipped).
cudaError_t launch_copy_back_f32(const float *src, float *dst, int64_t count, const PassStats *stats, int q,
                                 int grid, cudaStream_t s);
// Interleaved doubles -> floats in a layout (round to nearest), and back (exact).
cudaError_t launch_narrow(const double *aos, float *dst, int64_t n, int layout, int grid, cudaStream_t s);
cudaError_t launch_widen(const float *src, double *aos, int64_t n, int layout, int grid, cudaStream_t s);

// Ghost exchange of a domain-decomposed mesh: the listed nodes' coordinates
// (interleaved out / in, 2k doubles) from the current array, or into both
// arrays; an id outside [0, n) sets *bad and is skipped.  inv (caller's id ->
// internal id) maps the ids of a renumbered mesh; NULL when it is not.
cudaError_t launch_gather_nodes(const double *xy, int layout, int64_t n, const int32_t *idx, int64_t k,
                                const uint32_t *inv, double *out, unsigned *bad, int grid, cudaStream_t s);
cudaError_t launch_scatter_nodes(double *xy0, double *xy1, int layout, int64_t n, const int32_t *idx, int64_t k,
                                 const uint32_t *inv, const double *in, unsigned *bad, int grid, cudaStream_t s);

// A renumbered mesh (Form B: colour classes contiguous; Form A: nodes grouped
// by loop length inside windows of ids).  Coordinates are
// doubles or, with f32, floats, in the layout; perm maps a new id to the
// caller's.
// dst[k] = src[perm[k]]
cudaError_t launch_permute_coords(const double *src, double *dst, int layout, bool f32, int64_t n,
                                  const uint32_t *perm, int grid, cudaStream_t s);
// dst_aos (interleaved doubles, the caller's numbering)[perm[k]] = src[k]
cudaError_t launch_unpermute_to_aos(const double *src, int layout, bool f32, int64_t n, const uint32_t *perm,
                                    double *dst_aos, int grid, cudaStream_t s);
// dst[k] = src_aos (interleaved doubles, the caller's numbering)[perm[k]], rounded to floats with f32
cudaError_t launch_permute_from_aos(const double *src_aos, int layout, bool f32, int64_t n, const uint32_t *perm,
                                    double *dst, int grid, cudaStream_t s);
// dst[perm[k]] = src[k]
cudaError_t launch_unpermute_u8(const uint8_t *src, int64_t n, const uint32_t *perm, uint8_t *dst, int grid,
                                cudaStream_t s);

// Layout conversions on the device (SoA <-> interleaved).
cudaError_t launch_soa_to_aos(const double *soa, double *aos, int64_t n, int grid, cudaStream_t s);
cudaError_t launch_aos_to_soa(const double *aos, double *soa, int64_t n, int grid, cudaStream_t s);

}  // namespace sls
