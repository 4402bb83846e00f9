// sz_serve.cu -- in-situ serving loop (continuous batching).
#include "sz_ctx.h"

extern "C" {
sz_status sz_serve_start(sz_ctx* ctx, int slots) { (void)ctx; (void)slots; return SZ_ERR_UNSUPPORTED; }
sz_status sz_serve_submit(sz_ctx* ctx, const sz_request* req, uint64_t* ticket) { (void)ctx; (void)req; (void)ticket; return SZ_ERR_UNSUPPORTED; }
sz_status sz_serve_poll(sz_ctx* ctx, uint64_t ticket, sz_result* res) { (void)ctx; (void)ticket; (void)res; return SZ_ERR_UNSUPPORTED; }
sz_status sz_serve_stop(sz_ctx* ctx) { (void)ctx; return SZ_OK; }
}
