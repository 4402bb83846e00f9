/*
 * sz_gb300.h -- C ABI of the GB300 (sm_103a) SZ-LV compressor.
 *
 * The library compresses 1D float32 particle arrays with an error bound, as in
 * "In-Depth Exploration of Single-Snapshot Lossy Compression Techniques for
 * N-Body Simulations" (arXiv 1711.03888).  The problem statement is Sec. III:
 * every reconstructed value x'_i satisfies |x_i - x'_i| <= eb_abs, where the
 * bound is absolute or relative to the value range R = max - min.  The method
 * is SZ-LV (Sec. IV-A): last-value prediction on an integer lattice of step
 * D ~ 2*eb_abs, quantization into 2^16 codes, and Huffman coding of the codes.
 * For molecular dynamics (Sec. IV-B) the coordinates can first be reordered
 * by a segment-wise partial radix sort of their R-index (best_tradeoff mode).
 *
 * Conventions for every call:
 *   - Pointers named d_* are CUDA device pointers; h_* are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Calls only enqueue work on `stream` and return.  Sizes that the device
 *     computes (compressed bytes, element counts) are written through the
 *     caller's host pointers by sz_sync(), which also reports device-side
 *     errors.  The pointers must stay valid until that sz_sync().
 *   - A context is not thread-safe and owns one workspace: issue its calls
 *     from one host thread, on one stream at a time (use one context per
 *     concurrent stream).
 *   - No call aborts, traps or prints.  Each returns an sz_status; a device
 *     error is latched in the context and returned by the next sz_sync().
 *   - The caller owns every input and output buffer; the context owns its
 *     workspace (device memory it allocates and grows on demand).
 *
 * Stream format: a 160-byte header followed by the codebook, chunk tables,
 * sub-stream bit lengths, escape records and the Huffman payload.  No stream
 * is longer than sz_max_compressed_bytes(n).
 */
#ifndef SZ_GB300_H
#define SZ_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sz_ctx sz_ctx;

typedef enum {
    SZ_OK = 0,
    SZ_ERR_ARG = 1,          /* invalid argument (NULL, bad bound, bad parameters) */
    SZ_ERR_NOMEM = 2,        /* workspace allocation failed */
    SZ_ERR_CAPACITY = 3,     /* output buffer too small; required size reported */
    SZ_ERR_CORRUPT = 4,      /* malformed or truncated stream */
    SZ_ERR_CUDA = 5,         /* a CUDA runtime call failed */
    SZ_ERR_TIMEOUT = 6,      /* a bounded device wait expired */
    SZ_ERR_UNSUPPORTED = 7,  /* stream parameters this decoder does not handle */
    SZ_ERR_BUSY = 8          /* serving: no free slot or over the memory budget */
} sz_status;

/* Sec. III: absolute bound, or bound relative to the value range R. */
typedef enum { SZ_EB_ABS = 0, SZ_EB_REL = 1 } sz_eb_kind;

/* Sec. V: the three molecular-dynamics modes.  SZ_MODE_LV = best_speed (SZ-LV),
 * SZ_MODE_LV_PRX = best_tradeoff (SZ-LV-PRX), SZ_MODE_CPC2000 =
 * best_compression (SZ-CPC2000: CPC2000 on the coordinates, SZ-LV on the
 * other fields in the same order; see sz_compress_snapshot). */
typedef enum { SZ_MODE_LV = 0, SZ_MODE_LV_PRX = 1, SZ_MODE_CPC2000 = 2 } sz_mode;

/* Sec. III: the six particle fields. */
typedef enum {
    SZ_FIELD_XX = 0, SZ_FIELD_YY = 1, SZ_FIELD_ZZ = 2,
    SZ_FIELD_VX = 3, SZ_FIELD_VY = 4, SZ_FIELD_VZ = 5, SZ_FIELD_OTHER = 6
} sz_field;

/* Sec. IV-A: the predictor on the lattice.  SZ_PRED_LV = last value
 * (SZ-LV, delta = q_i - q_{i-1}); SZ_PRED_LCF = the original SZ's linear
 * curve fitting (delta = q_i - 2 q_{i-1} + q_{i-2}).  The stream records it
 * (header byte 43: 1 or 2); decoders accept both. */
typedef enum { SZ_PRED_DEFAULT = 0, SZ_PRED_LV = 1, SZ_PRED_LCF = 2 } sz_predictor;

/* Tuning parameters; a NULL pointer or a zero field selects the default.
 *   chunk_elems    elements per chunk: 2048, 4096, 8192 or 16384
 *                  (0 = the fixed rule from n: 2048 up to 2^16 elements,
 *                  else 4096; sz_compress_batch measures instead, see
 *                  sz_ctx_set_autotune).
 *   sub_elems      elements per sub-stream; must be chunk_elems / 64 (or 0).
 *   segment        MD mode: elements per sorted segment (Table 4), 1..65536
 *                  (0 = 16384).
 *   ignored_digits MD mode: 3-bit R-index digits ignored by the sort
 *                  (Table 5), 0..21 (the default 6 applies when segment is 0
 *                  too; set segment explicitly to request 0).
 *   predictor      an sz_predictor (0 = SZ_PRED_LV).  SZ_PRED_LCF runs the
 *                  per-array kernels: sz_compress_batch takes those arrays
 *                  one by one.
 *   key_fields     MD best_tradeoff mode: an sz_key_fields, the fields the
 *                  R-index is built from (0 = SZ_KEY_XYZ). */
typedef struct {
    uint32_t chunk_elems;
    uint32_t sub_elems;
    uint32_t segment;
    uint32_t ignored_digits;
    uint32_t predictor;
    uint32_t key_fields;
} sz_params;

/* Sec. IV-C, Fig. 3, Table 6: the R-index of the best_tradeoff reordering from
 * the coordinates (SZ_KEY_XYZ, Fig. 3a), the velocities (SZ_KEY_V: fields
 * 3..5 must be VX, VY, VZ; 3-bit digits) or all six (SZ_KEY_XYZV, Fig. 3b:
 * one bit of each of xx, yy, zz, vx, vy, vz per 6-bit digit, xx leading, at
 * most 10 bits per axis kept; ignored_digits then counts 6-bit digits, 0..10). */
typedef enum { SZ_KEY_XYZ = 0, SZ_KEY_V = 1, SZ_KEY_XYZV = 2 } sz_key_fields;

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the serving loop may admit at once (0 = no cap).  The workspace grows
 * with the largest array seen.  Errors: SZ_ERR_ARG (NULL ctx), SZ_ERR_CUDA,
 * SZ_ERR_NOMEM. */
sz_status sz_ctx_create(sz_ctx** ctx, int device, size_t hbm_budget_bytes);

/* Synchronize the context's device work and free the context and its workspace. */
sz_status sz_ctx_destroy(sz_ctx* ctx);

/* Largest stream any call can produce for n elements: 160 + 16*ceil(n/4). */
size_t sz_max_compressed_bytes(size_t n);

/* Compress d_in[0..n) (float32, device) into d_out (device, out_cap bytes).
 * Sec. III / IV-A: eb is absolute (SZ_EB_ABS) or relative to the value range
 * of the finite elements (SZ_EB_REL); it must be finite and >= 0.  n < 2^32.
 * On sz_sync(), *out_bytes holds the stream size, or the required size when
 * the call failed with SZ_ERR_CAPACITY (then d_out holds no valid stream).
 * Errors now: SZ_ERR_ARG; at sz_sync(): SZ_ERR_CAPACITY, SZ_ERR_TIMEOUT. */
sz_status sz_compress(sz_ctx* ctx, const float* d_in, size_t n, double eb, sz_eb_kind kind,
                      const sz_params* params, void* d_out, size_t out_cap, size_t* out_bytes,
                      void* stream);

/* Decompress a stream (device, in_bytes) into d_out (device, room for n_cap
 * floats).  Sec. III: every finite element is within the stream's eb_abs of
 * the original; non-finite elements come back bit-exact.  On sz_sync(),
 * *n_out holds the element count.  Errors at sz_sync(): SZ_ERR_CORRUPT
 * (malformed stream; no read leaves the in_bytes buffer), SZ_ERR_CAPACITY
 * (n_cap too small), SZ_ERR_UNSUPPORTED (sub-stream count other than 64). */
sz_status sz_decompress(sz_ctx* ctx, const void* d_in, size_t in_bytes, float* d_out, size_t n_cap,
                        size_t* n_out, void* stream);

/* Compress k independent arrays (the per-rank fields of a snapshot; Sec. V
 * compresses each in-memory array independently).  Arrays may have different
 * sizes and bounds; each stream is byte-identical to sz_compress on that
 * array with the same chunk size (the autotuner below may pick another chunk
 * size than sz_compress's fixed rule).  Arrays are processed together so
 * per-array fixed costs overlap: one CUDA graph per batch shape, replayed on
 * later calls.  Arguments are host arrays of k entries; out_bytes[i] is set
 * by sz_sync(). */
sz_status sz_compress_batch(sz_ctx* ctx, int k, const float* const* d_in, const size_t* n,
                            const double* eb, sz_eb_kind kind, const sz_params* params,
                            void* const* d_out, const size_t* out_cap, size_t* out_bytes,
                            void* stream);

/* Autotuning of the batched form.  When params leave chunk_elems and
 * sub_elems at 0 (and the predictor is LV), sz_compress_batch picks the chunk
 * size of each size class of arrays (n <= 2^16, <= 2^20, < 2^22, < 2^26, and
 * larger) and the item sizes of its persistent kernel by measurement: the
 * first time a class (or a batch shape) is seen, it compresses the batch --
 * or its first arrays, up to 2^30 elements -- with each candidate chunk size
 * (2048, 4096, 8192, 16384) into the caller's output buffers, decodes the
 * result into a temporary buffer, times both on the device with CUDA events
 * and keeps the fastest round trip.  The choice is cached in the context, so
 * later calls replay it; a tuning call synchronizes `stream` and allocates,
 * so make it outside stream capture.  Streams stay byte-identical to
 * sz_compress of the same array at the chosen chunk size (the header records
 * it).  sz_ctx_set_autotune(ctx, 0) switches the tuner off: the fixed rule
 * (2048 up to 2^16 elements, else 4096) then applies, as in sz_compress.
 * Errors: SZ_ERR_ARG (NULL ctx). */
sz_status sz_ctx_set_autotune(sz_ctx* ctx, int on);

/* What the autotuner chose for arrays of n elements (host struct).
 *   chunk_elems        the tuned chunk size of n's size class, 0 if not tuned yet
 *   fixed_chunk_elems  the fixed rule's chunk size for n
 *   class_lo, class_hi the size class, in elements (inclusive)
 *   trial_ms[j]        device ms of the trial round trip with chunk size
 *                      2048 << j (0 = not run or failed)
 *   range_tile, quant_group, tile_trial_ms[j]
 *                      the persistent kernel's item sizes (range elements,
 *                      quantize chunks) for the last tuned batch shape and the
 *                      compression ms of each candidate pair (0 if none)
 * Errors: SZ_ERR_ARG (NULL pointer). */
typedef struct {
    uint32_t chunk_elems;
    uint32_t fixed_chunk_elems;
    uint64_t class_lo, class_hi;
    float trial_ms[4];
    uint32_t range_tile, quant_group;
    float tile_trial_ms[4];
} sz_tuning;
sz_status sz_batch_tuning(sz_ctx* ctx, size_t n, sz_tuning* out);

/* Decompress k streams; each result equals sz_decompress of that stream. */
sz_status sz_decompress_batch(sz_ctx* ctx, int k, const void* const* d_in, const size_t* in_bytes,
                              float* const* d_out, const size_t* n_cap, size_t* n_out, void* stream);

/* Host-memory forms (Sec. I / Sec. III: in-situ compression of the arrays a
 * simulation holds in its own memory).  Same arguments as the batch calls,
 * but every data pointer (h_in, h_out) is HOST memory that the caller owns;
 * page-locked memory (cudaHostAlloc / cudaHostRegister) lets the copies run
 * asynchronously, pageable memory works but serializes them with the host.
 * The library stages the arrays through device memory of its own (two slots
 * of groups of consecutive arrays, each group at least 64 MiB of input):
 * copy-in of one group, the kernels of the previous one and the copy-out of
 * the one before run concurrently on two internal copy streams and `stream`.
 * Each stream (compress) and each array (decompress) is byte-identical to
 * sz_compress / sz_decompress of the same data.
 *
 * Both calls are SYNCHRONOUS: they return when every output is in host
 * memory, ending with sz_sync(ctx, stream) (which also delivers results of
 * earlier calls on `stream`) and returning its status.
 *
 * sz_compress_host: out_bytes[i] = stream size; when it exceeds out_cap[i]
 *   nothing is written to h_out[i] and the call returns SZ_ERR_CAPACITY.
 * sz_decompress_host: n_out[i] = element count from the stream's header;
 *   a stream of more than n_cap[i] elements writes nothing to h_out[i] and
 *   the call returns SZ_ERR_CAPACITY; a malformed stream returns
 *   SZ_ERR_CORRUPT (outputs of the call then undefined).
 * Errors: SZ_ERR_ARG (NULL arrays, bad bound, n >= 2^32), SZ_ERR_NOMEM
 * (staging), SZ_ERR_CUDA, and the device errors of sz_sync. */
sz_status sz_compress_host(sz_ctx* ctx, int k, const float* const* h_in, const size_t* n, const double* eb,
                           sz_eb_kind kind, const sz_params* params, void* const* h_out,
                           const size_t* out_cap, size_t* out_bytes, void* stream);
sz_status sz_decompress_host(sz_ctx* ctx, int k, const void* const* h_in, const size_t* in_bytes,
                             float* const* h_out, const size_t* n_cap, size_t* n_out, void* stream);

/* Molecular-dynamics snapshot (Sec. IV-B).  fields[0..2] must be XX, YY, ZZ;
 * further fields (velocities) follow the same reordering.  mode SZ_MODE_LV
 * compresses each field in stored order; SZ_MODE_LV_PRX first reorders every
 * field by one permutation: R-index keys from the lattice coordinates of the
 * three positions (Fig. 3a), stably sorted by key >> 3p within consecutive
 * segments (Tables 4-5).  No index array is stored (Sec. IV-B), so the
 * streams decode to the reordered arrays.  d_perm (device, n uint32, may be
 * NULL) receives the permutation: position j holds original index perm[j].
 * SZ_MODE_CPC2000 (Sec. II CPC2000 steps 1-4, Sec. IV-B SZ-CPC2000): all n
 * particles are stably sorted by the full R-index key (lossless: the lattice
 * coordinates must fit 21 bits per axis, else SZ_ERR_UNSUPPORTED at
 * sz_sync); d_out[0] (out_cap[0] >= sz_cpc_max_bytes(n)) receives ONE stream
 * holding all three coordinates -- key differences in Rice code, per block of
 * 4096 particles -- and d_out[1], d_out[2] are not written (out_bytes 0, may
 * be NULL); fields 3.. get SZ-LV streams in the sorted order.  Decode the
 * coordinate stream with sz_decompress_cpc, the others with sz_decompress. */
sz_status sz_compress_snapshot(sz_ctx* ctx, int nfields, const sz_field* fields,
                               const float* const* d_in, size_t n, const double* eb, sz_eb_kind kind,
                               sz_mode mode, const sz_params* params, void* const* d_out,
                               const size_t* out_cap, size_t* out_bytes, uint32_t* d_perm,
                               void* stream);

/* Largest SZ-CPC2000 coordinate stream for n particles. */
size_t sz_cpc_max_bytes(size_t n);

/* Decode an SZ-CPC2000 coordinate stream (device, in_bytes, 16-byte aligned)
 * into d_out[0..2] (device x, y, z arrays with room for n_cap floats each),
 * in the stream's sorted particle order.  Every coordinate is within its
 * axis's eb_abs of the original (non-finite and verbatim values come back
 * bit-exact).  On sz_sync(), *n_out holds the particle count.  Errors at
 * sz_sync(): SZ_ERR_CORRUPT (malformed stream; no read leaves in_bytes),
 * SZ_ERR_CAPACITY (n_cap too small). */
sz_status sz_decompress_cpc(sz_ctx* ctx, const void* d_in, size_t in_bytes, float* const* d_out, size_t n_cap,
                            size_t* n_out, void* stream);

/* Wait for the context's work on `stream`, fill the pending host results
 * (out_bytes, n_out) and return the first device error since the last sync
 * (SZ_OK if none), then clear it. */
sz_status sz_sync(sz_ctx* ctx, void* stream);

/* Exercise the timeout path of the device-side waits.  Every wait in the
 * kernels (the encoder's look-back on the chunks before its own, the batched
 * kernel's wait for an earlier phase) polls a bounded number of times and
 * then latches SZ_ERR_TIMEOUT instead of hanging.  This call enqueues on
 * `stream` one warp that runs the encoder's look-back wait against a
 * predecessor chunk that never publishes its size, polling at most `spins`
 * times (1 .. 2^20, a short sleep between polls).  The wait runs out, the
 * kernel latches SZ_ERR_TIMEOUT and returns; the next sz_sync() reports and
 * clears it, and the context stays usable.  The paper has no counterpart: the
 * waits belong to this library's parallel encoder.  Errors now: SZ_ERR_ARG
 * (NULL ctx, spins out of range), SZ_ERR_CUDA. */
sz_status sz_check_wait_timeout(sz_ctx* ctx, uint32_t spins, void* stream);

/* Human-readable name of a status code (static string). */
const char* sz_status_string(sz_status s);

/* ---- compression without allocation -------------------------------------- */

/* The paper has no counterpart to this call; it serves callers that cannot
 * let a library allocate device memory -- for example an in-situ simulation
 * whose own pool owns the GPU's memory, or code running where a cudaMalloc
 * would stall other streams.  It produces the same stream as sz_compress with
 * default parameters, byte for byte, but needs no context and allocates
 * nothing: its scratch (array state, histogram, codeword table, per-chunk
 * tables, codebook work arrays, error word; about 5.9 MB) is one fixed array
 * in device memory that every GPU loading this library keeps until exit.
 *   - n may be at most 2^26 elements; larger n returns SZ_ERR_ARG.
 *   - The call is synchronous: it enqueues the kernels on `stream`, waits for
 *     them and sets *out_bytes (host) before returning; device errors come
 *     back as its return value (SZ_ERR_CAPACITY: out_cap too small, with the
 *     required size in *out_bytes).
 *   - Every call looks up the scratch array's device address (the first call
 *     on a device is also where the array is set up; make that first call
 *     before any stream capture) and re-arms the array's state with one small
 *     kernel ahead of its own, so a device whose context was reset, which
 *     moves and zero-fills the array, is handled like a fresh one.
 *   - All calls on a device share the one array, which keeps the previous
 *     call's contents.  Calls that overlap on the GPU (other host threads or
 *     streams) race on it and must be serialized by the caller. */
sz_status sz_compress_noalloc(const float* d_in, size_t n, double eb, sz_eb_kind kind, void* d_out,
                              size_t out_cap, size_t* out_bytes, void* stream);

/* ---- tracing: per-phase kernel timing ------------------------------------ */

/* Kernel phases of the path: range (a1), lattice + histogram (a2-a4),
 * codebook + layout (a5, a8), encode (a6-a7), decoder setup, decode
 * (a9-a11), MD reordering (R-index keys + segment sort + gather), the
 * batched persistent kernel, and the chunk-size pass of the batched form's
 * two-pass encoder (the per-array calls count it under encode). */
typedef enum {
    SZ_PHASE_RANGE = 0, SZ_PHASE_QUANT = 1, SZ_PHASE_CODEBOOK = 2, SZ_PHASE_ENCODE = 3,
    SZ_PHASE_DECODE_SETUP = 4, SZ_PHASE_DECODE = 5, SZ_PHASE_REORDER = 6, SZ_PHASE_BATCH = 7,
    SZ_PHASE_ENCODE_SIZES = 8, SZ_NUM_PHASES = 9
} sz_phase;

/* Enable (on != 0) or disable tracing.  While enabled, the context records a
 * CUDA event pair around every kernel it launches.  Enabling clears the
 * counters. */
sz_status sz_profile_enable(sz_ctx* ctx, int on);

/* Wait for the recorded events and return, for each of the first nphases
 * phases, the number of kernel launches and their summed device time in
 * milliseconds (host arrays of nphases entries).  Clears the counters. */
sz_status sz_profile_read(sz_ctx* ctx, uint64_t* launches, double* ms, int nphases);

/* ---- serving: continuous batching of compress / decompress requests ----
 *
 * The paper's in-situ setting (Sec. I, Sec. III): every simulation rank
 * compresses the snapshot data it holds in memory.  Here many ranks' requests
 * share one GPU.  A host thread owned by the context admits queued requests in
 * arrival order whenever one of `slots` is free and the request's device bytes
 * fit the context's budget (hbm_budget_bytes of sz_ctx_create), launches its
 * kernels on the slot's own stream, so that admitted requests overlap on the
 * device, and retires it when its completion event fires.  Each request runs
 * the same kernels as sz_compress / sz_decompress on a private workspace, so
 * its result is byte-identical to the plain call's. */

typedef enum { SZ_OP_COMPRESS = 0, SZ_OP_DECOMPRESS = 1 } sz_op;

/* One request.  Input buffers are device pointers owned by the caller and must
 * stay valid until the request completes.  For SZ_OP_COMPRESS: in = float data
 * of n elements, out = stream buffer of out_cap bytes.  For SZ_OP_DECOMPRESS:
 * in = stream of in_bytes, out = float buffer of n (capacity) elements.
 * out = NULL asks the service for the output buffer: it is taken from a device
 * arena of hbm_budget_bytes (compress: sz_max_compressed_bytes(n) bytes;
 * decompress: 4*n bytes), returned in sz_result.out and held against the
 * budget until sz_serve_release.  That needs a nonzero budget. */
typedef struct {
    sz_op op;
    const void* in;
    size_t n;
    size_t in_bytes;
    void* out;
    size_t out_cap;
    double eb;
    sz_eb_kind kind;
} sz_request;

typedef struct {
    sz_status status;     /* SZ_OK once done; SZ_ERR_BUSY while pending */
    size_t out_size;      /* stream bytes (compress) or elements (decompress) */
    double latency_s;     /* completion seen on the host - submit time */
    void* out;            /* the output buffer (the caller's or the service's) */
} sz_result;

typedef struct {
    uint64_t submitted, completed;
    uint32_t peak_inflight;   /* most requests on the device at once */
    uint32_t peak_queue;      /* longest wait queue */
    size_t peak_bytes;        /* most budget bytes held at once */
    uint64_t budget_waits;    /* admissions that waited for budget bytes */
} sz_serve_counters;

/* Start the serving loop: up to `slots` (1..64) requests in flight.  A request
 * holds in_bytes-or-4n input bytes, its output bytes and 2n bytes of code
 * workspace against the budget while it runs; a service-owned output stays
 * held until released.  Errors: SZ_ERR_ARG (bad slots, loop already running),
 * SZ_ERR_NOMEM (arena), SZ_ERR_CUDA. */
sz_status sz_serve_start(sz_ctx* ctx, int slots);

/* Queue a request; *ticket identifies it.  Returns SZ_ERR_ARG for a bad
 * request, SZ_ERR_BUSY if it could never fit the memory budget. */
sz_status sz_serve_submit(sz_ctx* ctx, const sz_request* req, uint64_t* ticket);

/* Non-blocking: fills *res and forgets the ticket once done; res->status is
 * SZ_ERR_BUSY while pending.  SZ_ERR_ARG for an unknown ticket. */
sz_status sz_serve_poll(sz_ctx* ctx, uint64_t ticket, sz_result* res);

/* As sz_serve_poll, but waits up to timeout_s seconds for completion. */
sz_status sz_serve_wait(sz_ctx* ctx, uint64_t ticket, double timeout_s, sz_result* res);

/* Return a service-owned output buffer (sz_result.out of an out = NULL
 * request) to the arena.  SZ_ERR_ARG if `out` is not such a buffer. */
sz_status sz_serve_release(sz_ctx* ctx, void* out);

/* Counters since sz_serve_start. */
sz_status sz_serve_stats(sz_ctx* ctx, sz_serve_counters* out);

/* Drain all queued requests, stop the loop and free the arena (service-owned
 * outputs not yet released become invalid). */
sz_status sz_serve_stop(sz_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SZ_GB300_H */
