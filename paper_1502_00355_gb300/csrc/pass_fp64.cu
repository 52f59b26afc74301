// pass_fp64.cu -- the plain Jacobi pass of Smart Laplacian smoothing with
// every step on the FP64 pipe, plus the small auxiliary kernels.
//
// One thread per node (grid-stride).  For a free node i the thread
//   1. sums its neighbours' coordinates in the stored summation order and
//      divides by the degree (Eq. 2, Form A: only pass-q coordinates);
//   2. evaluates alpha of every incident triangle with node i at its pass-q
//      position (q_old) and at the centre (q_new), keeping the minima
//      (Section 3.3.4 and the per-pass refresh of all qualities);
//   3. keeps the centre iff q_new >= q_old (strict: >), writes the node, and
//      contributes its squared move and acceptance to the pass statistics.
// The FP64 pipe of GB300 is narrow, so this kernel is the exact baseline and
// the fallback of the screened kernel, not the fast path.
#include "kernels.h"
#include "node_exact.cuh"

namespace sls {

namespace {

template <int LAYOUT>
__global__ void __launch_bounds__(1024) pass_fp64_kernel(PassArgs a)
{
    if (pass_is_skipped(a.stats, a.q, a.tol_active, a.thr_bits)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.stats[a.q].executed = 1u;

    unsigned long long best = 0ull, nacc = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every node, or (a colour class of Form B) the listed free nodes
    const int64_t cnt = a.order ? a.norder : (a.ranged ? a.count : a.n);
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += stride) {
        const int64_t i = a.order ? (int64_t)__ldg(a.order + j) : a.first + j;
        const uint32_t meta = __ldg(a.adj + __ldg(a.node_off + i));
        if (meta & kMetaFixed) {
            if (a.accept) a.accept[i] = 0;
            continue;
        }
        unsigned long long bits;
        bool ok, moved;
        exact_update<LAYOUT>(a, i, 0u, 0u, 0ull, 0ull, bits, ok, moved);
        best = bits > best ? bits : best;
        nacc += ok ? 1ull : 0ull;
    }
    block_reduce_stats(a.stats + a.q, best, nacc, 0ull);
}

__global__ void copy_back_kernel(const double2 *__restrict__ src, double2 *__restrict__ dst,
                                 int64_t n2, const PassStats *stats, int q)
{
    if (stats[q].executed == 0u) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n2; k += stride)
        dst[k] = __ldg(src + k);
}

__device__ __forceinline__ unsigned long long order_key(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

template <int LAYOUT>
__global__ void histogram_kernel(const double *xy, int64_t n, const int32_t *__restrict__ tri,
                                 int64_t m, int nbins, double lo, double hi,
                                 unsigned long long *counts, unsigned long long *qmin_key,
                                 double *qsum)
{
    extern __shared__ unsigned long long s_counts[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) s_counts[b] = 0ull;
    __syncthreads();
    unsigned long long kmin = ~0ull;
    double sum = 0.0;
    const double width = __dsub_rn(hi, lo);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += stride) {
        const double2 A = Coords<LAYOUT>::get(xy, n, __ldg(tri + 3 * t));
        const double2 B = Coords<LAYOUT>::get(xy, n, __ldg(tri + 3 * t + 1));
        const double2 Cc = Coords<LAYOUT>::get(xy, n, __ldg(tri + 3 * t + 2));
        const double q = alpha_fp64(A.x, A.y, B.x, B.y, Cc.x, Cc.y);
        const double f = floor(__dmul_rn(__ddiv_rn(__dsub_rn(q, lo), width), (double)nbins));
        int bin = f < 0.0 ? 0 : (f >= (double)nbins ? nbins - 1 : (int)f);
        atomicAdd(&s_counts[bin], 1ull);
        const unsigned long long k = order_key(q);
        kmin = k < kmin ? k : kmin;
        sum = __dadd_rn(sum, q);
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long k2 = __shfl_xor_sync(0xffffffffu, kmin, o);
        kmin = k2 < kmin ? k2 : kmin;
        sum = __dadd_rn(sum, __shfl_xor_sync(0xffffffffu, sum, o));
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicMin(qmin_key, kmin);
        atomicAdd(qsum, sum);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        if (s_counts[b]) atomicAdd(&counts[b], s_counts[b]);
}

__global__ void soa_to_aos_kernel(const double *__restrict__ soa, double2 *__restrict__ aos, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        aos[i] = make_double2(__ldg(soa + i), __ldg(soa + n + i));
}

__global__ void aos_to_soa_kernel(const double2 *__restrict__ aos, double *__restrict__ soa, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double2 v = __ldg(aos + i);
        soa[i] = v.x;
        soa[n + i] = v.y;
    }
}

}  // namespace

cudaError_t launch_pass_fp64(const PassArgs &a, int layout, int block, int grid, cudaStream_t s)
{
    if (layout == 0) pass_fp64_kernel<0><<<grid, block, 0, s>>>(a);
    else pass_fp64_kernel<1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int pass_fp64_occupancy(int layout, int block)
{
    int nb = 0;
    if (layout == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_fp64_kernel<0>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_fp64_kernel<1>, block, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_copy_back(const double *src, double *dst, int64_t n_doubles,
                             const PassStats *stats, int q, int grid, cudaStream_t s)
{
    copy_back_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const double2 *>(src),
                                         reinterpret_cast<double2 *>(dst), n_doubles / 2, stats, q);
    return cudaGetLastError();
}

cudaError_t launch_histogram(const double *xy, int layout, int64_t n, const int32_t *tri,
                             int64_t m, int nbins, double lo, double hi,
                             unsigned long long *counts, unsigned long long *qmin_key,
                             double *qsum, int grid, cudaStream_t s)
{
    const size_t smem = sizeof(unsigned long long) * (size_t)nbins;
    if (layout == 0)
        histogram_kernel<0><<<grid, 256, smem, s>>>(xy, n, tri, m, nbins, lo, hi, counts, qmin_key, qsum);
    else
        histogram_kernel<1><<<grid, 256, smem, s>>>(xy, n, tri, m, nbins, lo, hi, counts, qmin_key, qsum);
    return cudaGetLastError();
}

namespace {

// Coordinates of the listed nodes out of the current array (ghost exchange
// of a domain-decomposed mesh); an id outside [0, n) sets *bad and is skipped.
template <int LAYOUT>
__global__ void gather_nodes_kernel(const double *__restrict__ xy, int64_t n, const int32_t *__restrict__ idx,
                                    int64_t k, const uint32_t *__restrict__ inv, double2 *__restrict__ out,
                                    unsigned *bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += stride) {
        const int32_t i = __ldg(idx + t);
        if (i < 0 || (int64_t)i >= n) {
            atomicOr(bad, 1u);
            continue;
        }
        out[t] = Coords<LAYOUT>::get(xy, n, inv ? (int64_t)__ldg(inv + i) : (int64_t)i);
    }
}

// The listed nodes' coordinates written into both arrays of the ping-pong.
template <int LAYOUT>
__global__ void scatter_nodes_kernel(double *xy0, double *xy1, int64_t n, const int32_t *__restrict__ idx,
                                     int64_t k, const uint32_t *__restrict__ inv, const double2 *__restrict__ in,
                                     unsigned *bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k; t += stride) {
        const int32_t i = __ldg(idx + t);
        if (i < 0 || (int64_t)i >= n) {
            atomicOr(bad, 1u);
            continue;
        }
        const double2 v = __ldg(in + t);
        const int64_t j = inv ? (int64_t)__ldg(inv + i) : (int64_t)i;
        Coords<LAYOUT>::put(xy0, n, j, v);
        Coords<LAYOUT>::put(xy1, n, j, v);
    }
}

}  // namespace

cudaError_t launch_gather_nodes(const double *xy, int layout, int64_t n, const int32_t *idx, int64_t k,
                                const uint32_t *inv, double *out, unsigned *bad, int grid, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    if (layout == 0)
        gather_nodes_kernel<0><<<grid, 256, 0, s>>>(xy, n, idx, k, inv, reinterpret_cast<double2 *>(out), bad);
    else
        gather_nodes_kernel<1><<<grid, 256, 0, s>>>(xy, n, idx, k, inv, reinterpret_cast<double2 *>(out), bad);
    return cudaGetLastError();
}

cudaError_t launch_scatter_nodes(double *xy0, double *xy1, int layout, int64_t n, const int32_t *idx, int64_t k,
                                 const uint32_t *inv, const double *in, unsigned *bad, int grid, cudaStream_t s)
{
    if (k <= 0) return cudaSuccess;
    const double2 *v = reinterpret_cast<const double2 *>(in);
    if (layout == 0)
        scatter_nodes_kernel<0><<<grid, 256, 0, s>>>(xy0, xy1, n, idx, k, inv, v, bad);
    else
        scatter_nodes_kernel<1><<<grid, 256, 0, s>>>(xy0, xy1, n, idx, k, inv, v, bad);
    return cudaGetLastError();
}

namespace {

// Coordinates in a layout and an element type (double or float).
template <class T, int LAYOUT>
struct Pair;
template <class T>
struct Pair<T, 0> {
    static __device__ __forceinline__ void get(const T *p, int64_t, int64_t i, T &x, T &y)
    {
        x = p[2 * i];
        y = p[2 * i + 1];
    }
    static __device__ __forceinline__ void put(T *p, int64_t, int64_t i, T x, T y)
    {
        p[2 * i] = x;
        p[2 * i + 1] = y;
    }
};
template <class T>
struct Pair<T, 1> {
    static __device__ __forceinline__ void get(const T *p, int64_t n, int64_t i, T &x, T &y)
    {
        x = p[i];
        y = p[n + i];
    }
    static __device__ __forceinline__ void put(T *p, int64_t n, int64_t i, T x, T y)
    {
        p[i] = x;
        p[n + i] = y;
    }
};

// dst[k] = src[perm[k]] (same layout and type)
template <class T, int LAYOUT>
__global__ void permute_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t n,
                               const uint32_t *__restrict__ perm)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        T x, y;
        Pair<T, LAYOUT>::get(src, n, perm[k], x, y);
        Pair<T, LAYOUT>::put(dst, n, k, x, y);
    }
}

// dst (interleaved doubles, the caller's numbering)[perm[k]] = src[k] (exact widening of floats)
template <class T, int LAYOUT>
__global__ void unpermute_to_aos_kernel(const T *__restrict__ src, int64_t n, const uint32_t *__restrict__ perm,
                                        double2 *__restrict__ dst)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        T x, y;
        Pair<T, LAYOUT>::get(src, n, k, x, y);
        dst[perm[k]] = make_double2((double)x, (double)y);
    }
}

// dst[k] = src (interleaved doubles, the caller's numbering)[perm[k]], rounded to T
template <class T, int LAYOUT>
__global__ void permute_from_aos_kernel(const double2 *__restrict__ src, int64_t n, const uint32_t *__restrict__ perm,
                                        T *__restrict__ dst)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        const double2 v = src[perm[k]];
        Pair<T, LAYOUT>::put(dst, n, k, (T)v.x, (T)v.y);
    }
}

__global__ void unpermute_u8_kernel(const uint8_t *__restrict__ src, int64_t n, const uint32_t *__restrict__ perm,
                                    uint8_t *__restrict__ dst)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) dst[perm[k]] = src[k];
}

}  // namespace

cudaError_t launch_permute_coords(const double *src, double *dst, int layout, bool f32, int64_t n,
                                  const uint32_t *perm, int grid, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (f32) {
        const float *fs = reinterpret_cast<const float *>(src);
        float *fd = reinterpret_cast<float *>(dst);
        if (layout == 0) permute_kernel<float, 0><<<grid, 256, 0, s>>>(fs, fd, n, perm);
        else permute_kernel<float, 1><<<grid, 256, 0, s>>>(fs, fd, n, perm);
    } else {
        if (layout == 0) permute_kernel<double, 0><<<grid, 256, 0, s>>>(src, dst, n, perm);
        else permute_kernel<double, 1><<<grid, 256, 0, s>>>(src, dst, n, perm);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpermute_to_aos(const double *src, int layout, bool f32, int64_t n, const uint32_t *perm,
                                    double *dst_aos, int grid, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    double2 *d = reinterpret_cast<double2 *>(dst_aos);
    if (f32) {
        const float *f = reinterpret_cast<const float *>(src);
        if (layout == 0) unpermute_to_aos_kernel<float, 0><<<grid, 256, 0, s>>>(f, n, perm, d);
        else unpermute_to_aos_kernel<float, 1><<<grid, 256, 0, s>>>(f, n, perm, d);
    } else {
        if (layout == 0) unpermute_to_aos_kernel<double, 0><<<grid, 256, 0, s>>>(src, n, perm, d);
        else unpermute_to_aos_kernel<double, 1><<<grid, 256, 0, s>>>(src, n, perm, d);
    }
    return cudaGetLastError();
}

cudaError_t launch_permute_from_aos(const double *src_aos, int layout, bool f32, int64_t n, const uint32_t *perm,
                                    double *dst, int grid, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const double2 *v = reinterpret_cast<const double2 *>(src_aos);
    if (f32) {
        float *f = reinterpret_cast<float *>(dst);
        if (layout == 0) permute_from_aos_kernel<float, 0><<<grid, 256, 0, s>>>(v, n, perm, f);
        else permute_from_aos_kernel<float, 1><<<grid, 256, 0, s>>>(v, n, perm, f);
    } else {
        if (layout == 0) permute_from_aos_kernel<double, 0><<<grid, 256, 0, s>>>(v, n, perm, dst);
        else permute_from_aos_kernel<double, 1><<<grid, 256, 0, s>>>(v, n, perm, dst);
    }
    return cudaGetLastError();
}

cudaError_t launch_unpermute_u8(const uint8_t *src, int64_t n, const uint32_t *perm, uint8_t *dst, int grid,
                                cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    unpermute_u8_kernel<<<grid, 256, 0, s>>>(src, n, perm, dst);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double *soa, double *aos, int64_t n, int grid, cudaStream_t s)
{
    soa_to_aos_kernel<<<grid, 256, 0, s>>>(soa, reinterpret_cast<double2 *>(aos), n);
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double *aos, double *soa, int64_t n, int grid, cudaStream_t s)
{
    aos_to_soa_kernel<<<grid, 256, 0, s>>>(reinterpret_cast<const double2 *>(aos), soa, n);
    return cudaGetLastError();
}

}  // namespace sls
