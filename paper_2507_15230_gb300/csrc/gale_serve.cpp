// Serving path: consumer requests, batching, HBM-budgeted relation cache.
#include <cstring>

#include "gale_ctx.h"

namespace gale {
void serve_destroy(gale_ctx *ctx) { (void)ctx; }
}  // namespace gale

extern "C" {

gale_status gale_request(gale_ctx *ctx, int32_t cluster_id, uint32_t mask, int64_t timeout_ns, gale_view *out) {
    (void)ctx; (void)cluster_id; (void)mask; (void)timeout_ns; (void)out;
    gale::set_error("serving is not built yet");
    return GALE_ENOTFOUND;
}

gale_status gale_release(gale_ctx *ctx, gale_view *view) {
    (void)ctx; (void)view;
    return GALE_OK;
}

gale_status gale_serve_stats_get(gale_ctx *ctx, gale_serve_stats *out) {
    (void)ctx;
    if (out) memset(out, 0, sizeof(*out));
    return GALE_OK;
}

gale_status gale_autotune(gale_ctx *ctx, uint32_t mask) {
    (void)ctx; (void)mask;
    return GALE_OK;
}

}  // extern "C"
