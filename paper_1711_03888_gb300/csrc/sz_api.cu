// sz_api.cu -- C ABI of the GB300 SZ-LV compressor (declared in
// include/sz_gb300.h).  The context owns a device workspace (per-array state,
// histogram, encoder table, chunk tables, codebook scratch, decoder tables),
// a device error word and pinned result slots.  Calls enqueue kernels on the
// caller's stream; sz_sync() copies device-computed sizes to the caller's
// pointers and reports latched device errors.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <mutex>
#include <vector>
#include "../../include/sz_gb300.h"
#include "sz_internal.h"
#include "sz_ctx.h"

using namespace szg;

namespace szg {

static const uint32_t kChunkChoices[] = {2048u, 4096u, 8192u, 16384u};

// The fixed chunk-size rule (not measured at run time): a pure function of n,
// so streams are reproducible.  4096-element chunks (64-element sub-streams)
// let eight decoder teams share an SM; small arrays use 2048 to keep every SM
// busy.  The plain and served calls use it; the batched form's autotuner
// replaces it there (sz_batch.cu).
uint32_t tune_chunk(uint64_t n) {
    if (n <= (1ull << 16)) return 2048u;
    return 4096u;
}

uint32_t params_pred(const sz_params* p) { return (p && p->predictor == SZ_PRED_LCF) ? kPredLCF : kPredLV; }

sz_status resolve_params(const sz_params* p, uint64_t n, uint32_t* C, uint32_t* G) {
    if (p && p->predictor > (uint32_t)SZ_PRED_LCF) return SZ_ERR_ARG;
    uint32_t c = (p && p->chunk_elems) ? p->chunk_elems : tune_chunk(n);
    bool ok = false;
    for (uint32_t v : kChunkChoices) ok |= (v == c);
    if (!ok) return SZ_ERR_ARG;
    uint32_t g = c / kSubPerChunk;
    if (p && p->sub_elems && p->sub_elems != g) return SZ_ERR_ARG;
    *C = c;
    *G = g;
    return SZ_OK;
}

static sz_status cuda_status(cudaError_t e) { return e == cudaSuccess ? SZ_OK : SZ_ERR_CUDA; }

sz_status ctx_reserve(sz_ctx* ctx, int arrays, uint64_t max_chunks, uint64_t max_code_elems) {
    if (arrays <= ctx->cap_arrays && max_chunks <= ctx->cap_chunks && max_code_elems <= ctx->cap_codes) return SZ_OK;
    int na = arrays > ctx->cap_arrays ? arrays : ctx->cap_arrays;
    uint64_t nc = max_chunks > ctx->cap_chunks ? max_chunks : ctx->cap_chunks;
    uint64_t ncode = max_code_elems > ctx->cap_codes ? max_code_elems : ctx->cap_codes;
    if (nc < 1024) nc = 1024;
    ncode = (ncode + 16383u) & ~(uint64_t)16383u;
    // in-flight work may still use the old buffers
    if (cudaDeviceSynchronize() != cudaSuccess) return SZ_ERR_CUDA;
    ctx->free_workspace();
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += (b + 255) & ~(size_t)255; return o; };
    size_t o_state = take(sizeof(ArrayState) * na);
    size_t o_hist = take(sizeof(uint32_t) * kNumCodes * na);
    size_t o_enc = take(sizeof(uint32_t) * kNumCodes * na);
    size_t o_cesc = take(sizeof(uint32_t) * nc * na);
    size_t o_cst = take(sizeof(unsigned long long) * nc * na);
    size_t o_cb = take(sizeof(uint32_t) * kCbScratchWords * na);
    size_t o_lut = take(sizeof(uint32_t) * kLutWords * na);
    size_t o_bylen = take(sizeof(uint16_t) * 65536 * na);
    size_t o_codes = take(sizeof(uint16_t) * ncode * na);
    void* base = nullptr;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_NOMEM;
    }
    ctx->ws = (uint8_t*)base;
    ctx->ws_bytes = bytes;
    ctx->d_state = (ArrayState*)(ctx->ws + o_state);
    ctx->d_hist = (uint32_t*)(ctx->ws + o_hist);
    ctx->d_enc = (uint32_t*)(ctx->ws + o_enc);
    ctx->d_chunk_esc = (uint32_t*)(ctx->ws + o_cesc);
    ctx->d_chunk_status = (unsigned long long*)(ctx->ws + o_cst);
    ctx->d_cb = (uint32_t*)(ctx->ws + o_cb);
    ctx->d_lut = (uint32_t*)(ctx->ws + o_lut);
    ctx->d_bylen = (uint16_t*)(ctx->ws + o_bylen);
    ctx->d_codes = (uint16_t*)(ctx->ws + o_codes);
    ctx->cap_arrays = na;
    ctx->cap_chunks = nc;
    ctx->cap_codes = ncode;
    // arm the range accumulators
    std::vector<ArrayState> init(na);
    memset(init.data(), 0, sizeof(ArrayState) * na);
    for (auto& s : init) { s.acc_min = 0xffffffffu; s.acc_max = 0u; s.min_key = 0xffffffffu; }
    if (cudaMemcpy(ctx->d_state, init.data(), sizeof(ArrayState) * na, cudaMemcpyHostToDevice) != cudaSuccess)
        return SZ_ERR_CUDA;
    if (cudaMemset(ctx->d_chunk_status, 0, sizeof(unsigned long long) * nc * na) != cudaSuccess) return SZ_ERR_CUDA;
    return SZ_OK;
}

CompressArgs make_compress_args(sz_ctx* ctx, int slot, const float* in, uint64_t n, double eb, int kind,
                                uint32_t C, uint32_t G, uint32_t extra_flags, void* out, uint64_t cap) {
    CompressArgs a;
    memset(&a, 0, sizeof(a));
    a.in = in;
    a.out = (uint8_t*)out;
    a.n = n;
    a.out_cap = cap;
    a.eb = eb;
    a.eb_kind = kind;
    a.C = C;
    a.G = G;
    a.n_chunks = (uint32_t)((n + C - 1) / C);
    a.extra_flags = extra_flags;
    a.st = ctx->d_state + slot;
    a.hist = ctx->d_hist + (size_t)kNumCodes * slot;
    a.enc = ctx->d_enc + (size_t)kNumCodes * slot;
    a.chunk_esc = ctx->d_chunk_esc + ctx->cap_chunks * slot;
    a.chunk_status = ctx->d_chunk_status + ctx->cap_chunks * slot;
    a.cb_scratch = ctx->d_cb + kCbScratchWords * slot;
    a.err = ctx->d_err;
    a.codes = ctx->d_codes + ctx->cap_codes * slot;
    a.grid_div = ctx->grid_div;
    return a;
}

DecompressArgs make_decompress_args(sz_ctx* ctx, int slot, const void* in, uint64_t in_bytes, float* out,
                                    uint64_t n_cap) {
    DecompressArgs d;
    memset(&d, 0, sizeof(d));
    d.in = (const uint8_t*)in;
    d.in_bytes = in_bytes;
    d.out = out;
    d.n_cap = n_cap;
    d.st = ctx->d_state + slot;
    d.lut = ctx->d_lut + (size_t)kLutWords * slot;
    d.by_len = ctx->d_bylen + (size_t)65536 * slot;
    d.cb_scratch = ctx->d_cb + kCbScratchWords * slot;
    d.err = ctx->d_err;
    d.grid_div = ctx->grid_div;
    return d;
}

// queue a device->pinned copy of one state field and remember where it goes
sz_status queue_result(sz_ctx* ctx, const void* dsrc, size_t* dst, cudaStream_t s) {
    if (!dst) return SZ_OK;
    if (ctx->n_pending >= ctx->cap_pending) return SZ_ERR_CAPACITY;
    uint64_t* slot = ctx->h_res + ctx->n_pending;
    ctx->pend_dst[ctx->n_pending] = dst;
    ctx->n_pending++;
    return cuda_status(cudaMemcpyAsync(slot, dsrc, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
}

sz_status validate_compress(const float* d_in, size_t n, double eb, sz_eb_kind kind, void* d_out) {
    if ((n && !d_in) || !d_out || ((uintptr_t)d_out & 15u) || ((uintptr_t)d_in & 3u)) return SZ_ERR_ARG;
    if (!(eb >= 0.0) || eb > 1.7976931348623157e308 || (kind != SZ_EB_ABS && kind != SZ_EB_REL)) return SZ_ERR_ARG;
    if ((uint64_t)n >= (1ull << 32)) return SZ_ERR_ARG;
    return SZ_OK;
}

static cudaEvent_t prof_event(sz_ctx* ctx) {
    if (ctx->prof_used < ctx->ev_pool.size()) return ctx->ev_pool[ctx->prof_used++];
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    ctx->ev_pool.push_back(e);
    ctx->prof_used++;
    return e;
}

ProfScope::ProfScope(sz_ctx* c, int ph, cudaStream_t st) : ctx(c), s(st), phase(ph) {
    if (ctx->prof_on && (a = prof_event(ctx))) cudaEventRecord(a, s);
}
ProfScope::~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(ctx);
    if (!b) return;
    cudaEventRecord(b, s);
    ctx->prof.push_back({phase, a, b});
}

// The four launches of one array's compression (range, quantize + histogram,
// codebook + layout, encode) followed by the result copy.
sz_status enqueue_compress(sz_ctx* ctx, const CompressArgs& a, size_t* out_bytes, cudaStream_t s) {
    { ProfScope p(ctx, SZ_PHASE_RANGE, s); launch_range(&a, 1, s); }
    { ProfScope p(ctx, SZ_PHASE_QUANT, s); launch_quant(&a, 1, s); }
    { ProfScope p(ctx, SZ_PHASE_CODEBOOK, s); launch_codebook(&a, 1, s); }
    if (a.n) { ProfScope p(ctx, SZ_PHASE_ENCODE, s); launch_encode(&a, 1, s); }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return queue_result(ctx, &a.st->total_bytes, out_bytes, s);
}

sz_status enqueue_decompress(sz_ctx* ctx, const DecompressArgs& d, size_t* n_out, cudaStream_t s) {
    { ProfScope p(ctx, SZ_PHASE_DECODE_SETUP, s); launch_decode_setup(&d, 1, s); }
    { ProfScope p(ctx, SZ_PHASE_DECODE, s); launch_decode(&d, 1, s); }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return queue_result(ctx, &d.st->n_out, n_out, s);
}

}  // namespace szg

void sz_ctx::free_workspace() {
    if (ws) cudaFree(ws);
    ws = nullptr;
    ws_bytes = 0;
    cap_arrays = 0;
    cap_chunks = 0;
    cap_codes = 0;
}

extern "C" {

sz_status sz_ctx_create(sz_ctx** out, int device, size_t hbm_budget_bytes) {
    if (!out) return SZ_ERR_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    sz_ctx* ctx = new sz_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    ctx->cap_pending = 1 << 16;
    if (cudaMalloc(&ctx->d_err, 256) != cudaSuccess || cudaMemset(ctx->d_err, 0, 256) != cudaSuccess ||
        cudaMallocHost(&ctx->h_res, sizeof(uint64_t) * (ctx->cap_pending + 8)) != cudaSuccess) {
        cudaGetLastError();
        sz_ctx_destroy(ctx);
        return SZ_ERR_CUDA;
    }
    ctx->h_err = reinterpret_cast<uint32_t*>(ctx->h_res + ctx->cap_pending);
    ctx->pend_dst.resize(ctx->cap_pending);
    sz_status s = ctx_reserve(ctx, 1, 1024, 0);
    if (s != SZ_OK) { sz_ctx_destroy(ctx); return s; }
    *out = ctx;
    return SZ_OK;
}

sz_status sz_ctx_destroy(sz_ctx* ctx) {
    if (!ctx) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    sz_serve_stop(ctx);
    cudaDeviceSynchronize();
    ctx->free_workspace();
    ctx->free_extra();
    ctx->free_host();
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_res) cudaFreeHost(ctx->h_res);
    delete ctx;
    return SZ_OK;
}

size_t sz_max_compressed_bytes(size_t n) { return (size_t)kHeaderBytes + 16u * ((n + 3u) / 4u); }

sz_status sz_compress(sz_ctx* ctx, const float* d_in, size_t n, double eb, sz_eb_kind kind, const sz_params* params,
                      void* d_out, size_t out_cap, size_t* out_bytes, void* stream) {
    if (!ctx) return SZ_ERR_ARG;
    sz_status s = validate_compress(d_in, n, eb, kind, d_out);
    if (s != SZ_OK) return s;
    uint32_t C, G;
    if ((s = resolve_params(params, n, &C, &G)) != SZ_OK) return s;
    cudaSetDevice(ctx->device);
    if ((s = ctx_reserve(ctx, 1, (n + C - 1) / C, (uint64_t)((n + C - 1) / C) * C)) != SZ_OK) return s;
    CompressArgs a = make_compress_args(ctx, 0, d_in, n, eb, (int)kind, C, G, 0u, d_out, out_cap);
    a.pred = params_pred(params);
    return enqueue_compress(ctx, a, out_bytes, (cudaStream_t)stream);
}

sz_status sz_decompress(sz_ctx* ctx, const void* d_in, size_t in_bytes, float* d_out, size_t n_cap, size_t* n_out,
                        void* stream) {
    if (!ctx || !d_in || ((uintptr_t)d_in & 15u) || (n_cap && !d_out) || ((uintptr_t)d_out & 3u)) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    DecompressArgs d = make_decompress_args(ctx, 0, d_in, in_bytes, d_out, n_cap);
    return enqueue_decompress(ctx, d, n_out, (cudaStream_t)stream);
}

sz_status sz_compress_batch(sz_ctx* ctx, int k, const float* const* d_in, const size_t* n, const double* eb,
                            sz_eb_kind kind, const sz_params* params, void* const* d_out, const size_t* out_cap,
                            size_t* out_bytes, void* stream) {
    if (!ctx || k < 0 || (k && (!d_in || !n || !eb || !d_out || !out_cap))) return SZ_ERR_ARG;
    return szg::batch_compress(ctx, k, d_in, n, eb, kind, params, d_out, out_cap, out_bytes, (cudaStream_t)stream);
}

sz_status sz_decompress_batch(sz_ctx* ctx, int k, const void* const* d_in, const size_t* in_bytes, float* const* d_out,
                              const size_t* n_cap, size_t* n_out, void* stream) {
    if (!ctx || k < 0 || (k && (!d_in || !in_bytes || !d_out || !n_cap))) return SZ_ERR_ARG;
    return szg::batch_decompress(ctx, k, d_in, in_bytes, d_out, n_cap, n_out, (cudaStream_t)stream);
}

sz_status sz_sync(sz_ctx* ctx, void* stream) {
    if (!ctx) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e1 = cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e2 = cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), s);
    cudaError_t e3 = cudaStreamSynchronize(s);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        cudaGetLastError();
        ctx->n_pending = 0;
        return SZ_ERR_CUDA;
    }
    for (uint32_t i = 0; i < ctx->n_pending; ++i) *ctx->pend_dst[i] = (size_t)ctx->h_res[i];
    ctx->n_pending = 0;
    uint32_t err = *ctx->h_err;
    if (err & E_TIMEOUT) return SZ_ERR_TIMEOUT;
    if (err & E_CORRUPT) return SZ_ERR_CORRUPT;
    if (err & E_UNSUPPORTED) return SZ_ERR_UNSUPPORTED;
    if (err & E_CAPACITY) return SZ_ERR_CAPACITY;
    if (err) return SZ_ERR_CUDA;
    return SZ_OK;
}

sz_status sz_ctx_set_autotune(sz_ctx* ctx, int on) {
    if (!ctx) return SZ_ERR_ARG;
    ctx->autotune = on != 0;
    return SZ_OK;
}

sz_status sz_batch_tuning(sz_ctx* ctx, size_t n, sz_tuning* out) {
    if (!ctx || !out) return SZ_ERR_ARG;
    memset(out, 0, sizeof(*out));
    static const uint64_t lo[kTuneClasses] = {0, (1ull << 16) + 1, (1ull << 20) + 1, 1ull << 22, 1ull << 26};
    static const uint64_t hi[kTuneClasses] = {1ull << 16, 1ull << 20, (1ull << 22) - 1, (1ull << 26) - 1,
                                              (1ull << 32) - 1};
    const int c = tune_class(n);
    out->chunk_elems = ctx->tune_C[c];
    out->fixed_chunk_elems = tune_chunk(n);
    out->class_lo = lo[c];
    out->class_hi = hi[c];
    for (int j = 0; j < kTuneCands; ++j) {
        out->trial_ms[j] = ctx->tune_ms[c][j];
        out->tile_trial_ms[j] = ctx->tile_ms[j];
    }
    out->range_tile = ctx->tile_range;
    out->quant_group = ctx->tile_group;
    return SZ_OK;
}

sz_status sz_check_wait_timeout(sz_ctx* ctx, uint32_t spins, void* stream) {
    if (!ctx || spins < 1 || spins > (1u << 20)) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    // the status word sits in the error word's block, past the error word
    unsigned long long* status = reinterpret_cast<unsigned long long*>(ctx->d_err + 32);
    launch_wait_timeout(status, ctx->d_err, spins, stream);
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return SZ_OK;
}

sz_status sz_profile_enable(sz_ctx* ctx, int on) {
    if (!ctx) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (!ctx->prof.empty()) cudaEventSynchronize(ctx->prof.back().b);
    ctx->prof.clear();
    ctx->prof_used = 0;
    ctx->prof_on = on != 0;
    return SZ_OK;
}

sz_status sz_profile_read(sz_ctx* ctx, uint64_t* launches, double* ms, int nphases) {
    if (!ctx || nphases < 0 || (nphases && (!launches || !ms))) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    for (int i = 0; i < nphases; ++i) { launches[i] = 0; ms[i] = 0.0; }
    sz_status st = SZ_OK;
    if (!ctx->prof.empty() && cudaEventSynchronize(ctx->prof.back().b) != cudaSuccess) st = SZ_ERR_CUDA;
    for (auto& r : ctx->prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) { cudaGetLastError(); st = SZ_ERR_CUDA; continue; }
        if (r.phase < nphases) { launches[r.phase]++; ms[r.phase] += t; }
    }
    ctx->prof.clear();
    ctx->prof_used = 0;
    return st;
}

const char* sz_status_string(sz_status s) {
    switch (s) {
        case SZ_OK: return "ok";
        case SZ_ERR_ARG: return "invalid argument";
        case SZ_ERR_NOMEM: return "out of device memory";
        case SZ_ERR_CAPACITY: return "output buffer too small";
        case SZ_ERR_CORRUPT: return "corrupt stream";
        case SZ_ERR_CUDA: return "CUDA error";
        case SZ_ERR_TIMEOUT: return "device wait timed out";
        case SZ_ERR_UNSUPPORTED: return "unsupported stream parameters";
        case SZ_ERR_BUSY: return "busy";
    }
    return "unknown status";
}

}  // extern "C"
