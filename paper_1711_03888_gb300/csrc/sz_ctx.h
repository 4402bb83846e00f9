// sz_ctx.h -- the context object behind the opaque sz_ctx handle.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>
#include "../../include/sz_gb300.h"
#include "sz_internal.h"

struct sz_serve_state;

struct sz_ctx {
    int device = 0;
    size_t budget = 0;
    uint32_t grid_div = 1;              // share of the GPU the persistent launches take (1/grid_div)
    // workspace (one block of device memory, grown on demand)
    uint8_t* ws = nullptr;
    size_t ws_bytes = 0;
    int cap_arrays = 0;
    uint64_t cap_chunks = 0;
    szg::ArrayState* d_state = nullptr;
    uint32_t* d_hist = nullptr;
    uint32_t* d_enc = nullptr;
    uint32_t* d_chunk_esc = nullptr;
    unsigned long long* d_chunk_status = nullptr;
    uint32_t* d_cb = nullptr;
    uint32_t* d_lut = nullptr;
    uint16_t* d_bylen = nullptr;
    uint16_t* d_codes = nullptr;
    uint64_t cap_codes = 0;
    uint32_t* d_err = nullptr;
    // pinned result slots and where sz_sync delivers them
    uint64_t* h_res = nullptr;
    uint32_t* h_err = nullptr;
    std::vector<size_t*> pend_dst;
    uint32_t n_pending = 0, cap_pending = 0;
    // MD reordering buffers
    uint8_t* md = nullptr;
    size_t md_bytes = 0;
    // batched form: per-array slices of one pool
    uint8_t* batch_pool = nullptr;
    size_t batch_bytes = 0;
    size_t batch_layout_bytes = 0;
    uint32_t batch_k = 0;
    int batch_states_armed = 0;
    // cached CUDA graph of the last batch (plan copy + counter reset + persistent kernel)
    uint64_t bg_key = 0;
    std::vector<uint8_t> bg_ident;      // the bytes the cached graph was built from
    cudaGraph_t bg_graph = nullptr;
    cudaGraphExec_t bg_exec = nullptr;
    cudaEvent_t bg_done = nullptr;
    uint8_t* batch_host = nullptr;      // pinned plan staging
    size_t batch_host_bytes = 0;
    // batched decompression: per-stream state and tables, and the plan staging
    uint8_t* dbatch_pool = nullptr;
    size_t dbatch_bytes = 0;
    uint8_t* dbatch_host = nullptr;
    size_t dbatch_host_bytes = 0;
    cudaEvent_t dbatch_done = nullptr;
    // host-memory calls: copy streams, per-slot events (copy-in done, kernels
    // done, copy-out done), device staging and pinned per-array results
    cudaStream_t host_h2d = nullptr, host_d2h = nullptr;
    cudaEvent_t host_ev[2][3] = {};
    uint8_t* host_pool = nullptr;
    size_t host_pool_bytes = 0;
    uint64_t* host_pin = nullptr;
    size_t host_pin_cap = 0;
    // SZ-CPC2000: sort buffers and per-block tables
    uint8_t* cpc = nullptr;
    size_t cpc_bytes = 0;
    // batched-form autotuner: chosen chunk size per size class of arrays (0 =
    // not tuned yet) with the trial times of the candidates, and the
    // persistent kernel's item sizes for the last tuned batch shape
    int autotune = 1;
    uint32_t tune_C[szg::kTuneClasses] = {};
    float tune_ms[szg::kTuneClasses][szg::kTuneCands] = {};
    uint64_t tile_key = 0;
    uint32_t tile_range = 0, tile_group = 0;
    float tile_ms[szg::kTuneCands] = {};
    // serving loop
    sz_serve_state* serve = nullptr;
    // tracing: event pairs around launches
    bool prof_on = false;
    struct ProfRec { int phase; cudaEvent_t a, b; };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t prof_used = 0;

    void free_workspace();
    void free_extra();
    void free_host();
};

namespace szg {
// Records an event before a launch and after it when tracing is on.
struct ProfScope {
    sz_ctx* ctx;
    cudaStream_t s;
    int phase;
    cudaEvent_t a = nullptr;
    ProfScope(sz_ctx* c, int ph, cudaStream_t st);
    ~ProfScope();
};
uint32_t tune_chunk(uint64_t n);
int tune_class(uint64_t n);   // size class of the batched form's autotuner (0 .. kTuneClasses-1)
sz_status resolve_params(const sz_params* p, uint64_t n, uint32_t* C, uint32_t* G);
uint32_t params_pred(const sz_params* p);     // kPredLV or kPredLCF
size_t cpc_max_bytes(uint64_t n);
// R-index keys from six fields (xx, yy, zz, vx, vy, vz; Fig. 3b): per-axis
// lattice range into qrange (12 words, order-mapped min then max), then keys
// of at most 10 bits per axis, shifted right by 6p, into key_lo / key_hi with
// the index within the segment in idx.
struct Reorder6Args {
    const float* pos[6];
    const ArrayState* st[6];
    uint64_t n;
    uint32_t segment, p;
    unsigned long long* qrange;
    uint32_t* key_lo;
    uint32_t* key_hi;
    uint32_t* idx;
    uint32_t* any_hi;
};
void launch_rindex_keys6(const Reorder6Args& a, void* stream);
sz_status cpc_compress_coords(sz_ctx* ctx, const ReorderArgs& r, uint64_t n, void* d_out, size_t out_cap,
                              size_t* out_bytes, uint32_t* perm_out, cudaStream_t s);
sz_status ctx_reserve(sz_ctx* ctx, int arrays, uint64_t max_chunks, uint64_t max_code_elems);
CompressArgs make_compress_args(sz_ctx* ctx, int slot, const float* in, uint64_t n, double eb, int kind,
                                uint32_t C, uint32_t G, uint32_t extra_flags, void* out, uint64_t cap);
DecompressArgs make_decompress_args(sz_ctx* ctx, int slot, const void* in, uint64_t in_bytes, float* out,
                                    uint64_t n_cap);
sz_status queue_result(sz_ctx* ctx, const void* dsrc, size_t* dst, cudaStream_t s);
sz_status validate_compress(const float* d_in, size_t n, double eb, sz_eb_kind kind, void* d_out);
sz_status enqueue_compress(sz_ctx* ctx, const CompressArgs& a, size_t* out_bytes, cudaStream_t s);
sz_status enqueue_decompress(sz_ctx* ctx, const DecompressArgs& d, size_t* n_out, cudaStream_t s);
sz_status batch_compress(sz_ctx* ctx, int k, const float* const* d_in, const size_t* n, const double* eb,
                         sz_eb_kind kind, const sz_params* params, void* const* d_out, const size_t* out_cap,
                         size_t* out_bytes, cudaStream_t s);
sz_status batch_decompress(sz_ctx* ctx, int k, const void* const* d_in, const size_t* in_bytes, float* const* d_out,
                           const size_t* n_cap, size_t* n_out, cudaStream_t s);
}  // namespace szg
