// sz_snapshot.cu -- the molecular-dynamics snapshot modes (Sec. IV-B, Sec. V):
// best_speed (SZ-LV: every field compressed in stored order) and
// best_tradeoff (SZ-LV-PRX: every field reordered by one permutation -- the
// segment-wise partial radix sort of the coordinates' R-index -- and then
// compressed with SZ-LV).  best_compression (SZ-CPC2000) is not built.
#include <string.h>
#include <vector>
#include "sz_ctx.h"

using namespace szg;

void sz_ctx::free_extra() {
    if (md) cudaFree(md);
    md = nullptr;
    md_bytes = 0;
    if (batch_pool) cudaFree(batch_pool);
    batch_pool = nullptr;
    batch_bytes = 0;
    batch_layout_bytes = 0;
    batch_states_armed = 0;
    if (bg_exec) cudaGraphExecDestroy(bg_exec);
    if (bg_graph) cudaGraphDestroy(bg_graph);
    if (bg_done) cudaEventDestroy(bg_done);
    if (batch_host) cudaFreeHost(batch_host);
    bg_exec = nullptr;
    bg_graph = nullptr;
    bg_done = nullptr;
    batch_host = nullptr;
    batch_host_bytes = 0;
    bg_key = 0;
    bg_ident.clear();
    if (dbatch_pool) cudaFree(dbatch_pool);
    if (dbatch_host) cudaFreeHost(dbatch_host);
    if (dbatch_done) cudaEventDestroy(dbatch_done);
    dbatch_pool = nullptr;
    dbatch_bytes = 0;
    dbatch_host = nullptr;
    dbatch_host_bytes = 0;
    dbatch_done = nullptr;
}

namespace {

// MD workspace: qrange (64 B) | any_hi (64 B) | 6 u32 arrays of n | nfields float arrays of n
sz_status md_reserve(sz_ctx* ctx, uint64_t n, int nfields, uint8_t** base) {
    const size_t need = 256 + sizeof(uint32_t) * 6 * n + sizeof(float) * (size_t)nfields * n + 1024;
    if (need > ctx->md_bytes) {
        if (cudaDeviceSynchronize() != cudaSuccess) return SZ_ERR_CUDA;
        ctx->free_extra();
        void* p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
        ctx->md = (uint8_t*)p;
        ctx->md_bytes = need;
    }
    *base = ctx->md;
    return SZ_OK;
}

}  // namespace

extern "C" sz_status sz_compress_snapshot(sz_ctx* ctx, int nfields, const sz_field* fields, const float* const* d_in,
                                          size_t n, const double* eb, sz_eb_kind kind, sz_mode mode,
                                          const sz_params* params, void* const* d_out, const size_t* out_cap,
                                          size_t* out_bytes, uint32_t* d_perm, void* stream) {
    if (!ctx || nfields < 1 || !d_in || !eb || !d_out || !out_cap) return SZ_ERR_ARG;
    if (mode != SZ_MODE_LV && mode != SZ_MODE_LV_PRX && mode != SZ_MODE_CPC2000) return SZ_ERR_ARG;
    const bool cpc = mode == SZ_MODE_CPC2000;
    cudaStream_t s = (cudaStream_t)stream;
    cudaSetDevice(ctx->device);
    for (int f = 0; f < nfields; ++f) {
        // best_compression writes all three coordinates to d_out[0]
        sz_status st = validate_compress(d_in[f], n, eb[f], kind, (cpc && (f == 1 || f == 2)) ? d_out[0] : d_out[f]);
        if (st != SZ_OK) return st;
    }
    uint32_t C, G;
    sz_status st = resolve_params(params, n, &C, &G);
    if (st != SZ_OK) return st;
    if (mode == SZ_MODE_LV) {
        if (d_perm) return SZ_ERR_ARG;   // no reordering, no permutation
        for (int f = 0; f < nfields; ++f) {
            st = sz_compress(ctx, d_in[f], n, eb[f], kind, params, d_out[f], out_cap[f],
                             out_bytes ? &out_bytes[f] : nullptr, stream);
            if (st != SZ_OK) return st;
        }
        return SZ_OK;
    }
    // ---- best_tradeoff (SZ-LV-PRX) and best_compression (SZ-CPC2000) -----------
    if (nfields < 3 || !fields || fields[0] != SZ_FIELD_XX || fields[1] != SZ_FIELD_YY || fields[2] != SZ_FIELD_ZZ)
        return SZ_ERR_ARG;
    // the fields the R-index is built from (Fig. 3): coordinates, velocities or all six
    const uint32_t keyf = params ? params->key_fields : (uint32_t)SZ_KEY_XYZ;
    if (keyf > (uint32_t)SZ_KEY_XYZV || (cpc && keyf != SZ_KEY_XYZ)) return SZ_ERR_ARG;
    if (keyf != SZ_KEY_XYZ &&
        (nfields < 6 || fields[3] != SZ_FIELD_VX || fields[4] != SZ_FIELD_VY || fields[5] != SZ_FIELD_VZ))
        return SZ_ERR_ARG;
    const int ax0 = keyf == SZ_KEY_V ? 3 : 0, nax = keyf == SZ_KEY_XYZV ? 6 : 3;
    // best_compression: keys of one segment with no ignored digits (a full sort follows)
    const uint32_t S = cpc ? (uint32_t)(n ? n : 1) : (params && params->segment) ? params->segment : 16384u;
    const uint32_t p = cpc ? 0u : (params && (params->segment || params->ignored_digits)) ? params->ignored_digits : 6u;
    if ((!cpc && S > 65536u) || p > (keyf == SZ_KEY_XYZV ? 10u : 21u)) return SZ_ERR_ARG;
    if ((st = ctx_reserve(ctx, ax0 + nax, (n + C - 1) / C, (uint64_t)((n + C - 1) / C) * C)) != SZ_OK) return st;
    uint8_t* md = nullptr;
    if ((st = md_reserve(ctx, n, nfields, &md)) != SZ_OK) return st;

    // a1 on the key fields (state slot = field index)
    for (int ax = ax0; ax < ax0 + nax; ++ax) {
        CompressArgs a = make_compress_args(ctx, ax, d_in[ax], n, eb[ax], (int)kind, C, G, 0u, d_out[ax], out_cap[ax]);
        ProfScope pr(ctx, SZ_PHASE_RANGE, s);
        launch_range(&a, 1, s);
    }
    ReorderArgs r;
    memset(&r, 0, sizeof(r));
    for (int ax = 0; ax < 3; ++ax) {
        r.pos[ax] = d_in[ax0 + ax];
        r.eb[ax] = eb[ax0 + ax];
        r.st[ax] = ctx->d_state + ax0 + ax;
    }
    r.n = n;
    r.eb_kind = (int)kind;
    r.segment = S;
    r.p = p;
    r.qrange = (unsigned long long*)md;
    r.any_hi = (uint32_t*)(md + 64);
    uint32_t* arr = (uint32_t*)(md + 256);
    r.key_lo = arr;
    r.key_hi = arr + n;
    r.idx = arr + 2 * n;
    r.tmp_k = arr + 3 * n;
    r.tmp_v = arr + 4 * n;
    r.perm = arr + 5 * n;
    r.err = ctx->d_err;
    float* permuted = (float*)(arr + 6 * n);
    const unsigned long long init[8] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    if (cudaMemcpyAsync(r.qrange, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(r.any_hi, 0, sizeof(uint32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    if (cpc) {
        // the coordinates: one SZ-CPC2000 stream in d_out[0]; the permutation into r.perm
        ProfScope pr(ctx, SZ_PHASE_REORDER, s);
        launch_rindex_keys(r, s);
        if ((st = cpc_compress_coords(ctx, r, n, d_out[0], out_cap[0], out_bytes ? &out_bytes[0] : nullptr, r.perm,
                                      s)) != SZ_OK)
            return st;
        if (out_bytes) out_bytes[1] = out_bytes[2] = 0;
        for (int f = 3; f < nfields; ++f) launch_gather(d_in[f], permuted + (size_t)f * n, r.perm, n, s);
    } else {
        ProfScope pr(ctx, SZ_PHASE_REORDER, s);
        if (keyf == SZ_KEY_XYZV) {
            Reorder6Args r6;
            memset(&r6, 0, sizeof(r6));
            for (int ax = 0; ax < 6; ++ax) {
                r6.pos[ax] = d_in[ax];
                r6.st[ax] = ctx->d_state + ax;
            }
            r6.n = n;
            r6.segment = S;
            r6.p = p;
            r6.qrange = (unsigned long long*)(md + 128);
            r6.key_lo = r.key_lo;
            r6.key_hi = r.key_hi;
            r6.idx = r.idx;
            r6.any_hi = r.any_hi;
            const unsigned long long init6[12] = {~0ull, ~0ull, ~0ull, ~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
            if (cudaMemcpyAsync(r6.qrange, init6, sizeof(init6), cudaMemcpyHostToDevice, s) != cudaSuccess) {
                cudaGetLastError();
                return SZ_ERR_CUDA;
            }
            launch_rindex_keys6(r6, s);
        } else {
            launch_rindex_keys(r, s);
        }
        launch_segment_sort(r, s);
        for (int f = 0; f < nfields; ++f) launch_gather(d_in[f], permuted + (size_t)f * n, r.perm, n, s);
    }
    if (d_perm && n &&
        cudaMemcpyAsync(d_perm, r.perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    // SZ-LV on every reordered field (best_compression: the fields after the
    // coordinates); streams carry the reordered flag
    for (int f = cpc ? 3 : 0; f < nfields; ++f) {
        CompressArgs a = make_compress_args(ctx, 0, permuted + (size_t)f * n, n, eb[f], (int)kind, C, G,
                                            kFlagReordered, d_out[f], out_cap[f]);
        a.pred = params_pred(params);
        if ((st = enqueue_compress(ctx, a, out_bytes ? &out_bytes[f] : nullptr, s)) != SZ_OK) return st;
    }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return SZ_OK;
}
