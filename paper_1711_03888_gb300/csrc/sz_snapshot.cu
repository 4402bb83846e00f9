// sz_snapshot.cu -- MD snapshot modes (Sec. IV-B / V: best_speed, best_tradeoff).
#include "sz_ctx.h"

using namespace szg;

void sz_ctx::free_extra() {
    if (md) cudaFree(md);
    md = nullptr;
    md_bytes = 0;
}

extern "C" sz_status sz_compress_snapshot(sz_ctx* ctx, int nfields, const sz_field* fields, const float* const* d_in,
                                          size_t n, const double* eb, sz_eb_kind kind, sz_mode mode,
                                          const sz_params* params, void* const* d_out, const size_t* out_cap,
                                          size_t* out_bytes, uint32_t* d_perm, void* stream) {
    if (!ctx || nfields < 1 || !d_in || !eb || !d_out || !out_cap) return SZ_ERR_ARG;
    if (mode == SZ_MODE_CPC2000) return SZ_ERR_UNSUPPORTED;
    if (mode != SZ_MODE_LV) return SZ_ERR_UNSUPPORTED;
    (void)fields; (void)d_perm;
    for (int f = 0; f < nfields; ++f) {
        sz_status s = sz_compress(ctx, d_in[f], n, eb[f], kind, params, d_out[f], out_cap[f],
                                  out_bytes ? &out_bytes[f] : nullptr, stream);
        if (s != SZ_OK) return s;
    }
    return SZ_OK;
}
