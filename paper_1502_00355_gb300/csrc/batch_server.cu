// batch_server.cu -- batched and served forms (placeholders until built).
#include "api_common.h"

using namespace sls;

extern "C" {

sls_status sls_batch_create(sls_mesh *const *, int32_t, const int32_t *, const double *,
                            const sls_options *, sls_batch **out)
{
    if (out) *out = nullptr;
    return fail(SLS_ERR_INVALID, "batched form not available in this build");
}
sls_status sls_batch_smooth(sls_batch *, sls_info *) { return fail(SLS_ERR_INVALID, "no batch"); }
sls_status sls_batch_get_coords(const sls_batch *, int32_t, double *) { return fail(SLS_ERR_INVALID, "no batch"); }
sls_status sls_batch_reset(sls_batch *) { return fail(SLS_ERR_INVALID, "no batch"); }
sls_status sls_batch_destroy(sls_batch *) { return SLS_OK; }
sls_status sls_server_create(size_t, int32_t, const sls_options *, sls_server **out)
{
    if (out) *out = nullptr;
    return fail(SLS_ERR_INVALID, "served form not available in this build");
}
sls_status sls_submit(sls_server *, const double *, int64_t, const int32_t *, int64_t, const uint8_t *,
                      int32_t, double, uint64_t *) { return fail(SLS_ERR_INVALID, "no server"); }
sls_status sls_wait(sls_server *, uint64_t, double, double *, sls_info *) { return fail(SLS_ERR_INVALID, "no server"); }
sls_status sls_server_stats(const sls_server *, double *, double *, double *, int64_t *) { return fail(SLS_ERR_INVALID, "no server"); }
sls_status sls_server_destroy(sls_server *) { return SLS_OK; }

}
