// sz_batch.cu -- many arrays per call (the per-rank fields of a snapshot).
// Each array's stream is byte-identical to sz_compress on that array.
#include <string.h>
#include "sz_ctx.h"

namespace szg {

sz_status batch_compress(sz_ctx* ctx, int k, const float* const* d_in, const size_t* n, const double* eb,
                         sz_eb_kind kind, const sz_params* params, void* const* d_out, const size_t* out_cap,
                         size_t* out_bytes, cudaStream_t s) {
    cudaSetDevice(ctx->device);
    uint64_t maxc = 0, maxcode = 0;
    for (int i = 0; i < k; ++i) {
        sz_status st = validate_compress(d_in[i], n[i], eb[i], kind, d_out[i]);
        if (st != SZ_OK) return st;
        uint32_t C, G;
        if ((st = resolve_params(params, n[i], &C, &G)) != SZ_OK) return st;
        uint64_t nc = (n[i] + C - 1) / C;
        if (nc > maxc) maxc = nc;
        if (nc * C > maxcode) maxcode = nc * C;
    }
    sz_status st = ctx_reserve(ctx, 1, maxc, maxcode);
    if (st != SZ_OK) return st;
    for (int i = 0; i < k; ++i) {
        uint32_t C, G;
        resolve_params(params, n[i], &C, &G);
        CompressArgs a = make_compress_args(ctx, 0, d_in[i], n[i], eb[i], (int)kind, C, G, 0u, d_out[i], out_cap[i]);
        if ((st = enqueue_compress(ctx, a, out_bytes ? &out_bytes[i] : nullptr, s)) != SZ_OK) return st;
    }
    return SZ_OK;
}

sz_status batch_decompress(sz_ctx* ctx, int k, const void* const* d_in, const size_t* in_bytes, float* const* d_out,
                           const size_t* n_cap, size_t* n_out, cudaStream_t s) {
    cudaSetDevice(ctx->device);
    for (int i = 0; i < k; ++i) {
        if (!d_in[i] || ((uintptr_t)d_in[i] & 15u) || (n_cap[i] && !d_out[i])) return SZ_ERR_ARG;
        DecompressArgs d = make_decompress_args(ctx, 0, d_in[i], in_bytes[i], d_out[i], n_cap[i]);
        sz_status st = enqueue_decompress(ctx, d, n_out ? &n_out[i] : nullptr, s);
        if (st != SZ_OK) return st;
    }
    return SZ_OK;
}

}  // namespace szg
