// sz_internal.h -- structures shared by the GB300 kernels and the C-ABI layer.
//
// Stream layout (version 1, little-endian), restated for the CUDA side:
//   header 160 B | symbols u16[m] | lengths u8[m] | chunk words u64[nc+1] |
//   chunk anchors i64[nc] | chunk escape bases u64[nc+1] |
//   sub-stream bit lengths u16[nc*C/G] | escapes 16 B each | payload u32[]
// Every section starts on a 16-byte boundary; padding bytes are zero.
#pragma once
#include <stdint.h>
#include <stddef.h>

namespace szg {

constexpr uint32_t kMagic = 0x564C5A53u;        // "SZLV"
constexpr uint32_t kVersion = 1;
constexpr uint32_t kHeaderBytes = 160;
constexpr int kMaxLen = 24;                       // longest codeword (bits)
constexpr int kRadius = 32768;                    // code = delta + radius, 0 = escape
constexpr int kNumCodes = 65536;
constexpr uint32_t kFlagRaw = 1u;
constexpr uint32_t kFlagReordered = 2u;
constexpr uint32_t kEscBytes = 16;
constexpr uint32_t kPredLV = 1;                   // header byte H_PRED: last value (Sec. IV-A)
constexpr uint32_t kPredLCF = 2;                  // linear curve fitting (Sec. IV-A, original SZ)
constexpr int kSubPerChunk = 64;                  // sub-streams per chunk on the GPU path
constexpr int kRangeBlocks = 1216;                // 8 x 152 SMs
constexpr int kLutBits = 12;                      // decoder direct-lookup width
constexpr int kLut2Bits = 16;                     // second level: codes of 13..16 bits by 16-bit prefix
constexpr uint32_t kLut2Max = 8192;               // second-level entries (further prefixes: limit walk)
constexpr uint32_t kLutWords = (1u << kLutBits) + kLut2Max;   // both levels, per array

// header byte offsets
constexpr int H_MAGIC = 0, H_VERSION = 4, H_HDRBYTES = 6, H_N = 8, H_EB = 16, H_D = 24,
              H_FLAGS = 28, H_C = 32, H_G = 36, H_M = 40, H_MAXLEN = 42, H_PRED = 43,
              H_NCHUNKS = 48, H_NSYM = 56, H_NESC = 64, H_PWORDS = 72, H_OFF = 80,
              H_TOTAL = 144;
enum { S_SYMS = 0, S_LENS, S_CWORD, S_ANCHOR, S_CESC, S_SUBLEN, S_ESC, S_PAYLOAD };

// error word bits (per context, set with atomicOr by kernels)
enum : uint32_t {
    E_CAPACITY = 1u, E_CORRUPT = 2u, E_TIMEOUT = 4u, E_UNSUPPORTED = 8u, E_INTERNAL = 16u
};

// Quantities every kernel derives the same way from the range (Sec. III).
struct LatticeParams {
    double eb_abs;      // absolute bound
    float D;            // lattice step: largest float <= 2*eb_abs
    float inv;          // ~1/D (candidate only)
    float thr_lo;       // RD32(D*(1/2 - 2^-20)): |x - qD| below -> q is certain
    float thr_hi;       // RU32(D*(1/2 + 2^-20)): |x - qD| above -> q is off by one
    float ebf;          // RD32(eb_abs): exact float form of the verbatim test
    int fast;           // D normal and in [2^-100, 2^100]
    int raw;            // D == 0: stream is a raw copy
};

// Per-array device state (workspace-resident).  Kernels of one call read and
// write it in stream order.
struct ArrayState {
    // range (set by the last range block)
    uint32_t min_key, max_key, any_finite, range_done;
    LatticeParams P;           // lattice parameters from the range (set with it)
    uint32_t acc_min, acc_max, acc_any, acc_blocks;   // accumulators, self-resetting
    // codebook / layout (set by the codebook kernel)
    uint64_t off[8];
    uint64_t n_escapes;
    uint64_t bound_bits;
    uint32_t n_used;
    uint32_t raw;
    uint32_t ticket;           // encoder chunk ticket (reset by the codebook kernel)
    uint32_t pred;             // decoder: predictor from the header (kPredLV / kPredLCF)
    uint64_t total_bytes;      // final stream size (set by the encoder)
    uint64_t n_out;            // decoder: element count from the header
    // decoder tables
    uint32_t first[kMaxLen + 2];
    uint32_t count[kMaxLen + 2];
    uint32_t base[kMaxLen + 2];
    uint32_t lim[kMaxLen + 2];   // left-justified end of each length's codes (24 bits)
    uint32_t dec_ok;
    uint32_t l2_lo;            // decoder: first 16-bit prefix of the second-level table
    uint32_t l2_n;             // decoder: its entries (0 = no second level)
    uint32_t max_cw;           // decoder: the largest chunk payload of the stream, in words
    uint32_t size_ticket;      // encoder pass 1 block ticket (reset by the codebook kernel)
    uint32_t cb_done;          // codebook: blocks done with their parallel build (re-armed by the range pass)
    uint32_t cb_ok[4];         // codebook: the build of h halvings fits the length limit
    uint32_t pad1[2];
};

// Arguments of one array's compression (passed by value to kernels).
struct CompressArgs {
    const float* in;
    uint8_t* out;
    uint64_t n;
    uint64_t out_cap;
    double eb;
    int eb_kind;                // 0 abs, 1 rel
    uint32_t C, G;
    uint32_t n_chunks;
    uint32_t extra_flags;
    ArrayState* st;
    uint32_t* hist;             // 65536
    uint32_t* enc;              // 65536: codeword << (32 - length) | escape << 5 | length
    uint32_t* chunk_esc;        // n_chunks: escapes per chunk
    unsigned long long* chunk_status;  // n_chunks: look-back words
    uint32_t* cb_scratch;       // codebook scratch (kCbScratchWords words)
    uint32_t* err;              // context error word
    uint16_t* codes;            // n_chunks*C u16 codes written by the quantizer, or null (encoder recomputes)
    uint32_t grid_div;          // persistent launches use 1/grid_div of the resident blocks (0, 1: all)
    uint32_t pred;              // kPredLCF: second-difference prediction (per-array path only); else LV
};

struct DecompressArgs {
    const uint8_t* in;
    uint64_t in_bytes;
    float* out;
    uint64_t n_cap;
    ArrayState* st;
    uint32_t* lut;              // kLutWords: 1 << kLutBits entries sym << 8 | len (0 = longer code),
                                //   then kLut2Max second-level entries for 16-bit prefixes l2_lo ..
    uint16_t* by_len;           // 65536: symbols in (length, symbol) order
    uint32_t* cb_scratch;
    uint32_t* err;
    uint32_t grid_div;          // the decode launch uses 1/grid_div of the SMs (0, 1: all)
};

// codebook scratch: 8 arrays of 65536 words and 5 of 131072 (layout in
// sz_codebook.cuh), rounded up; the decoder's setup uses the first 4 x 65536
constexpr size_t kCbScratchWords = 65536u * 20u;

// ---- host-side launchers (defined in the kernel files) ----
void launch_range(const CompressArgs* a, int k, void* stream);
void launch_quant(const CompressArgs* a, int k, void* stream);
void launch_codebook(const CompressArgs* a, int k, void* stream);
void launch_encode(const CompressArgs* a, int k, void* stream);
// one warp's look-back wait on a status word that nothing publishes (tests the
// timeout path); status: one device word, err: the context error word
void launch_wait_timeout(unsigned long long* status, uint32_t* err, uint32_t spins, void* stream);
void launch_decode_setup(const DecompressArgs* a, int k, void* stream);
void launch_decode(const DecompressArgs* a, int k, void* stream);
// Batched decompression: setup of all k streams (one block each) and the
// prefix of their decode units, then one launch over every unit.  d_args: k
// device entries; d_units: 2k words (units, then per-stream unit counters);
// d_uoff: k + 1 words.
void launch_decode_multi_setup(const DecompressArgs* d_args, uint32_t k, uint32_t* d_units, uint64_t* d_uoff,
                               void* stream);
void launch_decode_multi(const DecompressArgs* d_args, uint32_t k, uint32_t* d_units, const uint64_t* d_uoff,
                         void* stream);

// Batched form: one persistent launch over every array's work items.  The
// item sizes are tuned per batch shape; these are the defaults.
constexpr uint32_t kRangeTile = 1u << 16;   // elements per range item
constexpr uint32_t kQuantGroup = 8;         // chunks per quantize item

struct BatchCounters {          // per array, zeroed before the launch
    uint32_t range_done;        // range tiles finished
    uint32_t range_ready;       // 1 once the last tile published min / max
    uint32_t quant_done;        // quantize groups finished (histogram flushed)
    uint32_t cb_ready;          // 1 once the codebook and layout are written
};

struct BatchPlan {
    const CompressArgs* args;   // k (device)
    BatchCounters* cnt;         // k (device)
    const uint32_t* range_tiles;   // k
    const uint32_t* quant_groups;  // k
    const uint32_t* item_off;   // 4 x (k + 1): cumulative item offsets per phase, phase-major
    uint32_t k;
    uint32_t range_tile;        // elements per range item
    uint32_t quant_group;       // chunks per quantize item (quant_group * C <= 65535)
    uint32_t* next;             // item counter (zeroed before the launch)
    uint32_t* err;
};
void launch_batch_compress(const BatchPlan& plan, void* stream);
void batch_compress_config(void** func, unsigned* grid, unsigned* block, size_t* smem);

// Large arrays of a batch: one launch per phase over args[first .. first+count)
// of every group (the groups are contiguous; a group's arrays share C).
constexpr uint64_t kBatchLargeElems = 1ull << 22;
constexpr int kTuneClasses = 5;   // autotuner size classes: <=2^16, <=2^20, <2^22, <2^26, >=2^26 elements
constexpr int kTuneCands = 4;     // candidates per choice (chunk sizes 2048 .. 16384; item-size pairs)
constexpr uint32_t kBatchFewSmall = 304;   // at most this many small arrays: per-phase launches for all
struct MultiGroup {
    uint32_t first, count;      // arrays args[first .. first+count)
    uint32_t C;                 // their chunk size (2048 or 4096)
    uint32_t max_chunks;        // largest chunk count among them
};
struct MultiArgs {              // parameter of the per-phase kernels
    const CompressArgs* args;   // device
    uint32_t first;             // array of blockIdx.y == 0
};
struct KernelLaunch {           // one launch, for a graph node or a direct launch
    const void* func;
    unsigned grid[3], block[3];
    size_t smem;
    int phase;                  // tracing phase (sz_phase)
    MultiArgs args;
};
// Fills out[] with the per-phase launches (range, quantize, codebook, one
// encode per group), in dependency order; returns their count or -1.
int multi_compress_launches(const CompressArgs* d_args, const MultiGroup* groups, int ngroups, KernelLaunch* out,
                            int max_out);

// MD reordering (Sec. IV-B)
struct ReorderArgs {
    const float* pos[3];        // xx, yy, zz (device)
    uint64_t n;
    double eb[3];
    int eb_kind;
    uint32_t segment;           // S, 1 .. 65536
    uint32_t p;                 // ignored 3-bit digits, 0 .. 21
    const ArrayState* st[3];    // range state of the three coordinates
    unsigned long long* qrange; // 6: per-axis min (3) and max (3) lattice value, order-mapped
    uint32_t* key_lo;           // n: low word of key >> 3p (also sort scratch)
    uint32_t* key_hi;           // n: high word
    uint32_t* idx;              // n: index within the segment
    uint32_t* tmp_k;            // n: sort scratch
    uint32_t* tmp_v;            // n: sort scratch
    uint32_t* perm;             // n: position j holds original index perm[j]
    uint32_t* any_hi;           // 1: some key needs more than 32 bits
    uint32_t* err;
};
void launch_rindex_keys(const ReorderArgs& a, void* stream);
void launch_segment_sort(const ReorderArgs& a, void* stream);
void launch_gather(const float* src, float* dst, const uint32_t* perm, uint64_t n, void* stream);

}  // namespace szg
