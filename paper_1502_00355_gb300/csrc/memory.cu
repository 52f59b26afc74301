// memory.cu -- device memory of the library's handles.
//
// Every buffer a mesh, a build or a served job holds comes from one
// stream-ordered memory pool per device that the library owns
// (cudaMemPoolCreate), allocated and freed on the stream that uses it.  The
// pool keeps the memory that destroyed handles return, so a later handle of
// similar size reuses it at once instead of mapping new memory (cudaMalloc)
// and unmapping it again at the device-wide synchronisation of cudaFree.
// sls_trim_memory hands the kept memory back.  The pool is the library's
// own: the device's default pool, which other code in the process may use,
// is left as it is.
#include <mutex>

#include "api_common.h"

namespace sls {
namespace {

struct DevicePool {
    unsigned long long ctx = 0;  // the context the pool belongs to (0: none yet)
    cudaMemPool_t pool = nullptr;
};

std::mutex g_pool_mu;
DevicePool g_pools[64];

// The pool of the current device, made on first use and again after the
// device's context changed (cudaDeviceReset destroys pools).
cudaError_t current_pool(cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    DevicePool &P = g_pools[dev];
    if (P.pool && P.ctx == ctx && ctx != 0) {
        *out = P.pool;
        return cudaSuccess;
    }
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;  // keep freed memory until trimmed
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return e;
    }
    P.pool = pool;
    P.ctx = ctx;
    *out = pool;
    return cudaSuccess;
}

}  // namespace

cudaError_t pool_alloc(void **p, size_t bytes, cudaStream_t s)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = current_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes > 0 ? bytes : 1, pool, s);
}

void pool_free(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

}  // namespace sls

using namespace sls;

extern "C" sls_status sls_trim_memory(size_t keep_bytes)
{
    cudaMemPool_t pool = nullptr;
    cudaError_t e = current_pool(&pool);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // frees still queued on streams reach the pool
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, keep_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "sls_trim_memory");
    return SLS_OK;
}
