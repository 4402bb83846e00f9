// k_cpc.cu -- SZ-CPC2000 coordinates (best_compression mode; CPC2000 steps
// 1-4 of Sec. II, combined with SZ-LV for the other fields as in Sec. IV-B).
//
// Compression of the three coordinate arrays into one stream:
//   1. each coordinate on the SZ-LV lattice of its own bound (range kernels
//      of the compressor; verbatim rule as for SZ-LV);
//   2. the lossless R-index key of every particle (the MD key kernels with
//      one segment and no ignored digits; 3b <= 63 or E_UNSUPPORTED);
//   3. a stable device-wide LSD radix sort of (key, index): per 8-bit digit a
//      tile histogram, a digit-major scan and a scatter that ranks equal
//      digits in index order with warp match masks;
//   4. per block of 4096 sorted particles: the differences of adjacent keys
//      (0 for the first), the Rice parameter k of fewest bits (exact costs
//      for all 64 candidates, the smallest on ties), the bit length of each
//      of the 32 sub-streams of 128 particles, and the verbatim coordinates;
//      one block then lays out the stream and writes the header, and a pack
//      launch writes codewords (d >> k zero bits, a one bit, the low k bits
//      of d, MSB-first; each block's bits padded to whole words and owned by
//      one CUDA block) and exception records.
// Decompression: a setup block validates the header against in_bytes; one
// warp per coding block decodes its 32 sub-streams in two passes (sums, a
// warp scan, then keys -> lattice coordinates -> RN32(q D)); exception
// records are patched last.  Every payload read is bounds-checked.
#include <cuda_runtime.h>
#include <string.h>
#include "../../include/sz_gb300.h"
#include "sz_internal.h"
#include "sz_ctx.h"
#include "sz_device.cuh"

namespace szg {

namespace {

constexpr uint32_t kCpcMagic = 0x50435A53u;     // "SZCP"
constexpr uint32_t kCpcBlock = 4096;            // particles per coding block
constexpr uint32_t kCpcSubs = 32;               // sub-streams per coding block
constexpr uint32_t kCpcSubLen = kCpcBlock / kCpcSubs;
constexpr int kCpcThreads = 256;                // encode: 16 particles per thread
constexpr int kCpcPer = kCpcBlock / kCpcThreads;
constexpr uint32_t kTile = 4096;                // radix sort tile
constexpr int kSortT = 256;
constexpr int kDigits = 256;
// header byte offsets
constexpr int C_N = 8, C_EB = 16, C_D = 40, C_B = 52, C_QMIN = 56, C_BLOCK = 80, C_SUBS = 84, C_NB = 88, C_NE = 96,
              C_WORDS = 104, C_OFF = 112;
enum { T_FIRST = 0, T_WORDS, T_K, T_SUB, T_EXC, T_PAYLOAD };

struct CpcState {
    uint64_t n, nb, ne, words, total, cap;
    uint64_t off[6];
    long long qmin[3];
    double eb_abs[3];
    float D[3];
    uint32_t b, ok, raw[3];
    LatticeParams P[3];
};

struct CpcArgs {
    CpcState* st;
    const float* pos[3];
    const ArrayState* ast[3];           // range states of the coordinates (compression)
    const unsigned long long* qrange;   // per-axis lattice min / max, order-mapped
    const uint32_t* key_lo;
    const uint32_t* key_hi;
    unsigned long long* ka;             // sort buffers
    unsigned long long* kb;
    uint32_t* va;
    uint32_t* vb;
    uint32_t* counts;                   // kDigits * ntiles
    unsigned long long* dbase;          // kDigits
    uint64_t ntiles;
    unsigned long long* blk_first;      // nb
    uint32_t* blk_k;                    // nb
    unsigned long long* blk_words;      // nb + 1 (scanned in place)
    unsigned long long* blk_exc;        // nb + 1 (scanned in place)
    uint32_t* sub_off;                  // nb * kCpcSubs
    uint8_t* out;
    const uint8_t* in;
    uint64_t in_bytes;
    float* dst[3];
    uint64_t n_cap;
    uint32_t* err;
    uint32_t shift;                     // radix pass
};

__device__ __forceinline__ long long q_unorder64(unsigned long long u) { return (long long)(u ^ 0x8000000000000000ull); }

// remove the two bits between every kept bit (inverse of the 3-way spread)
__device__ __forceinline__ unsigned long long compact3(unsigned long long v) {
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v | (v >> 4)) & 0x100f00f00f00f00full;
    v = (v | (v >> 8)) & 0x1f0000ff0000ffull;
    v = (v | (v >> 16)) & 0x1f00000000ffffull;
    v = (v | (v >> 32)) & 0x1fffffull;
    return v;
}

__device__ __forceinline__ bool coord_verbatim(float x, const LatticeParams& P) {
    if (P.raw) return true;
    long long q;
    bool v;
    lattice_q(x, P, q, v);
    return v;
}

// ---- compression ----------------------------------------------------------------

// key width and lattice origin; (key, index) pairs for the sort
__global__ void cpc_params_kernel(CpcArgs a) {
    CpcState* st = a.st;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long umax = 0;
        for (int ax = 0; ax < 3; ++ax) {
            st->P[ax] = a.ast[ax]->P;
            st->D[ax] = st->P[ax].D;
            st->eb_abs[ax] = st->P[ax].eb_abs;
            st->raw[ax] = st->P[ax].raw;
            st->qmin[ax] = st->n ? q_unorder64(a.qrange[ax]) : 0;
            if (st->n) {
                const unsigned long long span = (unsigned long long)(q_unorder64(a.qrange[3 + ax]) - st->qmin[ax]);
                umax = umax > span ? umax : span;
            }
        }
        const uint32_t b = umax ? 64 - __clzll((long long)umax) : 0;
        st->b = b;
        st->ok = b <= 21;
        if (b > 21) raise_err(a.err, E_UNSUPPORTED);
    }
}

__global__ void cpc_pairs_kernel(CpcArgs a) {
    const uint64_t n = a.st->n;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        a.ka[i] = ((unsigned long long)a.key_hi[i] << 32) | a.key_lo[i];
        a.va[i] = (uint32_t)i;
    }
}

__device__ __forceinline__ bool pass_live(const CpcState* st, uint32_t shift) { return st->ok && shift < 3 * st->b; }

// radix pass, 1/3: digit counts of each tile, digit-major
__global__ void __launch_bounds__(kSortT) cpc_hist_kernel(CpcArgs a, const unsigned long long* k) {
    __shared__ uint32_t h[kDigits];
    if (!pass_live(a.st, a.shift)) return;
    const uint64_t n = a.st->n, t0 = (uint64_t)blockIdx.x * kTile;
    h[threadIdx.x] = 0;
    __syncthreads();
    for (uint64_t i = t0 + threadIdx.x; i < umin64(n, t0 + kTile); i += kSortT)
        atomicAdd(&h[(uint32_t)(k[i] >> a.shift) & 0xffu], 1u);
    __syncthreads();
    a.counts[(uint64_t)threadIdx.x * a.ntiles + blockIdx.x] = h[threadIdx.x];
}

// 2/3: exclusive scan over the tiles of one digit (block = digit), then of the digit totals
__global__ void __launch_bounds__(1024) cpc_scan_tiles_kernel(CpcArgs a) {
    __shared__ unsigned long long ws[33];
    __shared__ unsigned long long carry;
    if (!pass_live(a.st, a.shift)) return;
    uint32_t* c = a.counts + (uint64_t)blockIdx.x * a.ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < a.ntiles; b0 += 1024) {
        const uint64_t i = b0 + threadIdx.x;
        const unsigned long long v = i < a.ntiles ? c[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan<1024>(v, ws, &tot);
        if (i < a.ntiles) c[i] = (uint32_t)(carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.dbase[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kDigits) cpc_scan_digits_kernel(CpcArgs a) {
    __shared__ unsigned long long ws[33];
    if (!pass_live(a.st, a.shift)) return;
    unsigned long long tot;
    const unsigned long long v = a.dbase[threadIdx.x];
    const unsigned long long ex = block_exclusive_scan<kDigits>(v, ws, &tot);
    __syncthreads();
    a.dbase[threadIdx.x] = ex;
}

// 3/3: stable scatter.  The tile is taken 256 elements at a time in index
// order; inside a round an element's rank is its rank among equal digits of
// its warp (match mask) plus the counts of those digits in earlier warps of
// the round and earlier rounds of the tile.  A dead pass copies.
__global__ void __launch_bounds__(kSortT) cpc_scatter_kernel(CpcArgs a, const unsigned long long* k, const uint32_t* v,
                                                             unsigned long long* k2, uint32_t* v2) {
    __shared__ uint32_t wc[kSortT / 32][kDigits];
    __shared__ unsigned long long run[kDigits];
    const uint64_t n = a.st->n, t0 = (uint64_t)blockIdx.x * kTile, t1 = umin64(n, t0 + kTile);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (!pass_live(a.st, a.shift)) {
        for (uint64_t i = t0 + tid; i < t1; i += kSortT) {
            k2[i] = k[i];
            v2[i] = v[i];
        }
        return;
    }
    run[tid] = a.dbase[tid] + a.counts[(uint64_t)tid * a.ntiles + blockIdx.x];
    for (uint64_t r0 = t0; r0 < t1; r0 += kSortT) {
        for (int d = lane; d < kDigits; d += 32) wc[w][d] = 0;
        __syncthreads();
        const uint64_t i = r0 + tid;
        const bool live = i < t1;
        const unsigned long long key = live ? k[i] : 0ull;
        const uint32_t dg = live ? ((uint32_t)(key >> a.shift) & 0xffu) : kDigits;   // kDigits: no element
        const uint32_t peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t below = __popc(peers & ((1u << lane) - 1u));
        if (live && below == 0) wc[w][dg] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over the warps, and the round's total
        {
            uint32_t acc = 0;
            for (int ww = 0; ww < kSortT / 32; ++ww) {
                const uint32_t c = wc[ww][tid];
                wc[ww][tid] = acc;
                acc += c;
            }
            __syncthreads();
            if (live) {
                const unsigned long long pos = run[dg] + wc[w][dg] + below;
                k2[pos] = key;
                v2[pos] = v[i];
            }
            __syncthreads();
            run[tid] += acc;
        }
        __syncthreads();
    }
}

// per coding block: Rice parameter, sub-stream offsets, block words, exceptions
__global__ void __launch_bounds__(kCpcThreads) cpc_block_kernel(CpcArgs a, const unsigned long long* ks,
                                                                const uint32_t* perm) {
    __shared__ unsigned long long cost[64];
    __shared__ unsigned long long ws[kCpcThreads / 32 + 1];
    __shared__ uint32_t s_k;
    const CpcState* st = a.st;
    if (!st->ok) return;
    const uint64_t n = st->n, blk = blockIdx.x, j0 = blk * kCpcBlock;
    const uint32_t L = (uint32_t)umin64(kCpcBlock, n - j0);
    const int tid = threadIdx.x;
    unsigned long long d[kCpcPer];
    uint32_t exc = 0;
#pragma unroll
    for (int e = 0; e < kCpcPer; ++e) {
        const uint32_t i = tid * kCpcPer + e;
        d[e] = 0;
        if (i < L) {
            if (i) d[e] = ks[j0 + i] - ks[j0 + i - 1];
            const uint32_t o = perm[j0 + i];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) exc += coord_verbatim(__ldg(a.pos[ax] + o), st->P[ax]) ? 1u : 0u;
        }
    }
    if (tid < 64) cost[tid] = 0;
    __syncthreads();
    // exact bit counts for every k: sum (d >> k) + L (1 + k)
    for (int k = 0; k < 64; ++k) {
        unsigned long long s = 0;
#pragma unroll
        for (int e = 0; e < kCpcPer; ++e) s += d[e] >> k;
        s = warp_reduce_sum(s);
        if ((tid & 31) == 0 && s) atomicAdd(&cost[k], s);
    }
    __syncthreads();
    if (tid == 0) {
        int best = 0;
        unsigned long long bc = ~0ull;
        for (int k = 0; k < 64; ++k) {
            const unsigned long long c = cost[k] + (unsigned long long)L * (1u + k);
            if (c < bc) { bc = c; best = k; }
        }
        s_k = best;
    }
    __syncthreads();
    const uint32_t k = s_k;
    unsigned long long bits = 0;
#pragma unroll
    for (int e = 0; e < kCpcPer; ++e)
        if (tid * kCpcPer + e < L) bits += (d[e] >> k) + 1u + k;
    unsigned long long tot;
    const unsigned long long ex = block_exclusive_scan<kCpcThreads>(bits, ws, &tot);
    if ((tid % (kCpcSubLen / kCpcPer)) == 0) a.sub_off[blk * kCpcSubs + tid / (kCpcSubLen / kCpcPer)] = (uint32_t)ex;
    __syncthreads();
    unsigned long long etot;
    block_exclusive_scan<kCpcThreads>((unsigned long long)exc, ws, &etot);
    if (tid == 0) {
        a.blk_first[blk] = ks[j0];
        a.blk_k[blk] = k;
        a.blk_words[blk] = (tot + 31) / 32;
        a.blk_exc[blk] = etot;
    }
}

__device__ __forceinline__ uint64_t pad16d(uint64_t b) { return (b + 15u) & ~(uint64_t)15u; }

// one block: block word offsets, exception bases, layout, header, capacity
__global__ void __launch_bounds__(1024) cpc_layout_kernel(CpcArgs a) {
    __shared__ unsigned long long ws[33];
    __shared__ unsigned long long carry[2];
    __shared__ uint32_t s_ok;
    CpcState* st = a.st;
    if (!st->ok) return;
    const uint64_t nb = st->nb;
    if (threadIdx.x == 0) carry[0] = carry[1] = 0;
    __syncthreads();
    for (uint64_t b0 = 0; b0 < nb; b0 += 1024) {
        const uint64_t i = b0 + threadIdx.x;
        const unsigned long long w = i < nb ? a.blk_words[i] : 0ull, e = i < nb ? a.blk_exc[i] : 0ull;
        unsigned long long tw, te;
        const unsigned long long xw = block_exclusive_scan<1024>(w, ws, &tw);
        __syncthreads();
        const unsigned long long xe = block_exclusive_scan<1024>(e, ws, &te);
        if (i < nb) {
            a.blk_words[i] = carry[0] + xw;
            a.blk_exc[i] = carry[1] + xe;
        }
        __syncthreads();
        if (threadIdx.x == 0) { carry[0] += tw; carry[1] += te; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const uint64_t words = carry[0], ne = carry[1];
        a.blk_words[nb] = words;
        a.blk_exc[nb] = ne;
        uint64_t o = kHeaderBytes;
        st->off[T_FIRST] = o;   o = pad16d(o + 8 * nb);
        st->off[T_WORDS] = o;   o = pad16d(o + 8 * (nb + 1));
        st->off[T_K] = o;       o = pad16d(o + nb);
        st->off[T_SUB] = o;     o = pad16d(o + 4ull * kCpcSubs * nb);
        st->off[T_EXC] = o;     o = pad16d(o + 16 * ne);
        st->off[T_PAYLOAD] = o;
        st->words = words;
        st->ne = ne;
        st->total = o + 4 * words;
        s_ok = st->total <= st->cap;
        if (!s_ok) {
            raise_err(a.err, E_CAPACITY);
            st->ok = 0;
        }
    }
    __syncthreads();
    if (!s_ok) return;
    if (threadIdx.x == 0) {
        const uint64_t words = st->words, ne = st->ne, n = st->n;
        uint8_t* out = a.out;
        for (uint32_t i = 0; i < kHeaderBytes / 4; ++i) reinterpret_cast<uint32_t*>(out)[i] = 0u;
        *reinterpret_cast<uint32_t*>(out) = kCpcMagic;
        *reinterpret_cast<uint16_t*>(out + 4) = 1;
        *reinterpret_cast<uint16_t*>(out + 6) = (uint16_t)kHeaderBytes;
        *reinterpret_cast<uint64_t*>(out + C_N) = n;
        for (int ax = 0; ax < 3; ++ax) {
            *reinterpret_cast<double*>(out + C_EB + 8 * ax) = st->eb_abs[ax];
            *reinterpret_cast<float*>(out + C_D + 4 * ax) = st->D[ax];
            *reinterpret_cast<long long*>(out + C_QMIN + 8 * ax) = st->qmin[ax];
        }
        *reinterpret_cast<uint32_t*>(out + C_B) = st->b;
        *reinterpret_cast<uint32_t*>(out + C_BLOCK) = kCpcBlock;
        *reinterpret_cast<uint32_t*>(out + C_SUBS) = kCpcSubs;
        *reinterpret_cast<uint64_t*>(out + C_NB) = nb;
        *reinterpret_cast<uint64_t*>(out + C_NE) = ne;
        *reinterpret_cast<uint64_t*>(out + C_WORDS) = words;
        for (int s = 0; s < 6; ++s) *reinterpret_cast<uint64_t*>(out + C_OFF + 8 * s) = st->off[s];
        reinterpret_cast<unsigned long long*>(out + st->off[T_WORDS])[nb] = words;
        (void)ne;
    }
    // zero the padding bytes after each table section
    uint8_t* out = a.out;
    const uint64_t* off = st->off;
    const uint64_t used[5] = {off[T_FIRST] + 8 * nb, off[T_WORDS] + 8 * (nb + 1), off[T_K] + nb,
                              off[T_SUB] + 4ull * kCpcSubs * nb, off[T_EXC] + 16 * st->ne};
    for (int sct = 0; sct < 5; ++sct)
        for (uint64_t b = used[sct] + threadIdx.x; b < off[sct + 1]; b += blockDim.x) out[b] = 0;
}

// write `len` (1..64) bits of v, MSB-first, at bit `pos` of the payload
__device__ __forceinline__ void put_bits(uint32_t* words, uint64_t pos, unsigned long long v, uint32_t len) {
    while (len) {
        const uint32_t off = (uint32_t)(pos & 31u), room = 32u - off, take = len < room ? len : room;
        const uint32_t chunk = (uint32_t)((v >> (len - take)) & ((1ull << take) - 1ull));
        atomicOr(&words[pos >> 5], chunk << (room - take));
        pos += take;
        len -= take;
    }
}

// per coding block: tables, codewords, exception records (the block owns its words)
__global__ void __launch_bounds__(kCpcThreads) cpc_pack_kernel(CpcArgs a, const unsigned long long* ks,
                                                               const uint32_t* perm) {
    __shared__ unsigned long long ws[kCpcThreads / 32 + 1];
    const CpcState* st = a.st;
    if (!st->ok) return;
    const uint64_t n = st->n, nb = st->nb, blk = blockIdx.x, j0 = blk * kCpcBlock;
    const uint32_t L = (uint32_t)umin64(kCpcBlock, n - j0);
    const int tid = threadIdx.x;
    uint8_t* out = a.out;
    uint32_t* payload = reinterpret_cast<uint32_t*>(out + st->off[T_PAYLOAD]);
    const uint64_t wb = a.blk_words[blk], we = a.blk_words[blk + 1];
    const uint32_t k = a.blk_k[blk];
    for (uint64_t w = wb + tid; w < we; w += kCpcThreads) payload[w] = 0u;
    if (tid < (int)kCpcSubs)
        reinterpret_cast<uint32_t*>(out + st->off[T_SUB])[blk * kCpcSubs + tid] = a.sub_off[blk * kCpcSubs + tid];
    if (tid == 0) {
        reinterpret_cast<unsigned long long*>(out + st->off[T_FIRST])[blk] = a.blk_first[blk];
        out[st->off[T_K] + blk] = (uint8_t)k;
        reinterpret_cast<unsigned long long*>(out + st->off[T_WORDS])[blk] = wb;
    }
    (void)nb;
    unsigned long long d[kCpcPer];
    unsigned long long bits = 0;
    uint32_t exc = 0;
#pragma unroll
    for (int e = 0; e < kCpcPer; ++e) {
        const uint32_t i = tid * kCpcPer + e;
        d[e] = 0;
        if (i < L) {
            if (i) d[e] = ks[j0 + i] - ks[j0 + i - 1];
            bits += (d[e] >> k) + 1u + k;
            const uint32_t o = perm[j0 + i];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) exc += coord_verbatim(__ldg(a.pos[ax] + o), st->P[ax]) ? 1u : 0u;
        }
    }
    unsigned long long tot;
    unsigned long long pos = block_exclusive_scan<kCpcThreads>(bits, ws, &tot) + 32ull * wb;
    __syncthreads();          // the block's words are zero
#pragma unroll
    for (int e = 0; e < kCpcPer; ++e) {
        if (tid * kCpcPer + e >= L) break;
        pos += d[e] >> k;
        const unsigned long long low = k ? (d[e] & ((1ull << k) - 1ull)) : 0ull;
        put_bits(payload, pos, (1ull << k) | low, k + 1u);
        pos += k + 1u;
    }
    unsigned long long etot;
    const unsigned long long eoff = block_exclusive_scan<kCpcThreads>((unsigned long long)exc, ws, &etot);
    if (exc) {
        uint8_t* rec = out + st->off[T_EXC] + 16 * (a.blk_exc[blk] + eoff);
        for (int e = 0; e < kCpcPer; ++e) {
            const uint32_t i = tid * kCpcPer + e;
            if (i >= L) break;
            const uint32_t o = perm[j0 + i];
            for (int ax = 0; ax < 3; ++ax) {
                const float x = __ldg(a.pos[ax] + o);
                if (coord_verbatim(x, st->P[ax])) {
                    *reinterpret_cast<unsigned long long*>(rec) = j0 + i;
                    *reinterpret_cast<uint32_t*>(rec + 8) = (uint32_t)ax;
                    *reinterpret_cast<uint32_t*>(rec + 12) = __float_as_uint(x);
                    rec += 16;
                }
            }
        }
    }
}

// ---- decompression --------------------------------------------------------------

__device__ __forceinline__ uint64_t rd64c(const uint8_t* p) { return *reinterpret_cast<const uint64_t*>(p); }
__device__ __forceinline__ uint32_t rd32c(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

__global__ void cpc_setup_kernel(CpcArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    CpcState* st = a.st;
    const uint8_t* in = a.in;
    st->ok = 0;
    st->n = 0;
    uint32_t status = 0;
    if (a.in_bytes < kHeaderBytes || rd32c(in) != kCpcMagic || *reinterpret_cast<const uint16_t*>(in + 4) != 1 ||
        *reinterpret_cast<const uint16_t*>(in + 6) != kHeaderBytes) {
        status = E_CORRUPT;
    } else {
        const uint64_t n = rd64c(in + C_N), nb = rd64c(in + C_NB), ne = rd64c(in + C_NE), words = rd64c(in + C_WORDS);
        const uint32_t b = rd32c(in + C_B);
        uint64_t off[6];
        for (int s = 0; s < 6; ++s) off[s] = rd64c(in + C_OFF + 8 * s);
        bool bad = n >= (1ull << 32) || b > 21 || rd32c(in + C_BLOCK) != kCpcBlock || rd32c(in + C_SUBS) != kCpcSubs ||
                   nb != (n + kCpcBlock - 1) / kCpcBlock || ne > 3 * n || words > (1ull << 40);
        for (int s = 0; !bad && s < 6; ++s) bad = off[s] < kHeaderBytes || (off[s] & 15u) || (s && off[s] < off[s - 1]);
        if (!bad)
            bad = off[T_WORDS] - off[T_FIRST] < 8 * nb || off[T_K] - off[T_WORDS] < 8 * (nb + 1) ||
                  off[T_SUB] - off[T_K] < nb || off[T_EXC] - off[T_SUB] < 4ull * kCpcSubs * nb ||
                  off[T_PAYLOAD] - off[T_EXC] < 16 * ne || off[T_PAYLOAD] + 4 * words > a.in_bytes;
        if (bad) {
            status = E_CORRUPT;
        } else {
            st->n = n;
            st->nb = nb;
            st->ne = ne;
            st->words = words;
            st->b = b;
            for (int s = 0; s < 6; ++s) st->off[s] = off[s];
            for (int ax = 0; ax < 3; ++ax) {
                st->D[ax] = __uint_as_float(rd32c(in + C_D + 4 * ax));
                st->qmin[ax] = *reinterpret_cast<const long long*>(in + C_QMIN + 8 * ax);
            }
            if (n > a.n_cap) status = E_CAPACITY;
        }
    }
    if (status) raise_err(a.err, status);
    st->ok = status == 0;
}

struct BitIn {
    const uint32_t* p;
    uint64_t nwords, pos, end;
    __device__ __forceinline__ uint32_t peek32() const {
        const uint64_t w = pos >> 5;
        const uint32_t hi = w < nwords ? __ldg(p + w) : 0u, lo = w + 1 < nwords ? __ldg(p + w + 1) : 0u;
        return (uint32_t)(((((unsigned long long)hi << 32) | lo) << (pos & 31u)) >> 32);
    }
    // one Rice codeword; false past the block's end
    __device__ __forceinline__ bool rice(uint32_t k, unsigned long long& d) {
        unsigned long long zeros = 0;
        for (;;) {
            if (pos >= end) return false;
            const uint32_t v = peek32();
            if (v) {
                const uint32_t z = __clz(v);
                zeros += z;
                pos += z;
                break;
            }
            zeros += 32;
            pos += 32;
        }
        if (pos + 1 + k > end) return false;
        pos += 1;
        unsigned long long r = 0;
        if (k > 32) {
            r = (unsigned long long)peek32() << (k - 32);
            pos += 32;
            r |= peek32() >> (64 - k);
            pos += k - 32;
        } else if (k) {
            r = peek32() >> (32 - k);
            pos += k;
        }
        d = (zeros << k) | r;
        return true;
    }
};

// one warp per coding block (lane = sub-stream), grid-stride over the blocks
__global__ void __launch_bounds__(128) cpc_decode_kernel(CpcArgs a) {
    const CpcState* st = a.st;
    if (!st->ok) return;
    const uint8_t* in = a.in;
    const uint64_t n = st->n, nb = st->nb;
    const uint32_t* payload = reinterpret_cast<const uint32_t*>(in + st->off[T_PAYLOAD]);
    const int lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const long long qmin[3] = {st->qmin[0], st->qmin[1], st->qmin[2]};
    const float D[3] = {st->D[0], st->D[1], st->D[2]};
    for (uint64_t blk = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); blk < nb; blk += warps) {
        const uint64_t j0 = blk * kCpcBlock;
        const uint32_t L = (uint32_t)umin64(kCpcBlock, n - j0);
        const uint64_t wb = rd64c(in + st->off[T_WORDS] + 8 * blk), we = rd64c(in + st->off[T_WORDS] + 8 * (blk + 1));
        const uint32_t k = in[st->off[T_K] + blk];
        const uint32_t so = rd32c(in + st->off[T_SUB] + 4 * (blk * kCpcSubs + lane));
        const bool hdr_bad = wb > we || we > st->words || k > 63 || so > 32ull * (we - wb);
        if (__any_sync(0xffffffffu, hdr_bad)) {
            if (lane == 0) raise_err(a.err, E_CORRUPT);
            continue;
        }
        const uint32_t i0 = lane * kCpcSubLen, i1 = i0 + kCpcSubLen < L ? i0 + kCpcSubLen : L;
        BitIn br{payload, st->words, 32ull * wb + so, 32ull * we};
        unsigned long long sum = 0, d;
        bool bad = false;
        for (uint32_t i = i0; i < i1 && !bad; ++i) {
            if (br.rice(k, d)) sum += d; else bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            if (lane == 0) raise_err(a.err, E_CORRUPT);
            continue;
        }
        // exclusive warp scan of the sub-stream sums
        unsigned long long inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        unsigned long long key = rd64c(in + st->off[T_FIRST] + 8 * blk) + (inc - sum);
        br.pos = 32ull * wb + so;
        for (uint32_t i = i0; i < i1; ++i) {
            br.rice(k, d);
            key += d;
            const uint64_t j = j0 + i;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const long long q = (long long)compact3(key >> (2 - ax)) + qmin[ax];
                a.dst[ax][j] = recon_f(q, D[ax]);
            }
        }
    }
}

__global__ void cpc_exceptions_kernel(CpcArgs a) {
    const CpcState* st = a.st;
    if (!st->ok) return;
    const uint8_t* rec = a.in + st->off[T_EXC];
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < st->ne; e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t j = rd64c(rec + 16 * e);
        const uint32_t ax = rd32c(rec + 16 * e + 8);
        if (j >= st->n || ax > 2) {
            raise_err(a.err, E_CORRUPT);
            continue;
        }
        a.dst[ax][j] = __uint_as_float(rd32c(rec + 16 * e + 12));
    }
}

int sm_count_cpc() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// scratch of one compression or decompression of n particles
sz_status cpc_reserve(sz_ctx* ctx, uint64_t n, uint8_t** base, size_t* layout) {
    const uint64_t nt = (n + kTile - 1) / kTile, nb = (n + kCpcBlock - 1) / kCpcBlock;
    size_t o = 0;
    auto take = [&](size_t b) { size_t r = o; o += a256(b); return r; };
    layout[0] = take(sizeof(CpcState));
    layout[1] = take(8 * n);                        // ka
    layout[2] = take(8 * n);                        // kb
    layout[3] = take(4 * n);                        // va
    layout[4] = take(4 * n);                        // vb
    layout[5] = take(4ull * kDigits * (nt ? nt : 1));
    layout[6] = take(8 * kDigits);
    layout[7] = take(8 * nb);                       // blk_first
    layout[8] = take(4 * nb);                       // blk_k
    layout[9] = take(8 * (nb + 1));                 // blk_words
    layout[10] = take(8 * (nb + 1));                // blk_exc
    layout[11] = take(4ull * kCpcSubs * nb);        // sub_off
    if (o > ctx->cpc_bytes) {
        if (cudaDeviceSynchronize() != cudaSuccess) return SZ_ERR_CUDA;
        if (ctx->cpc) cudaFree(ctx->cpc);
        ctx->cpc = nullptr;
        ctx->cpc_bytes = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, o) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
        ctx->cpc = (uint8_t*)p;
        ctx->cpc_bytes = o;
    }
    *base = ctx->cpc;
    return SZ_OK;
}

}  // namespace

size_t cpc_max_bytes(uint64_t n) {
    const uint64_t nb = (n + kCpcBlock - 1) / kCpcBlock;
    return (size_t)(kHeaderBytes + 16 * 6 + 8 * nb + 8 * (nb + 1) + nb + 4ull * kCpcSubs * nb + 48 * n + 9 * n +
                    4 * nb + 64);
}

// Coordinates of an MD snapshot (range states in slots 0..2 already computed,
// keys of one segment with no ignored digits in r) into d_out; the
// permutation into perm_out (n words).
sz_status cpc_compress_coords(sz_ctx* ctx, const ReorderArgs& r, uint64_t n, void* d_out, size_t out_cap,
                              size_t* out_bytes, uint32_t* perm_out, cudaStream_t s) {
    uint8_t* base = nullptr;
    size_t lay[12];
    sz_status st = cpc_reserve(ctx, n, &base, lay);
    if (st != SZ_OK) return st;
    CpcArgs a;
    memset(&a, 0, sizeof(a));
    a.st = (CpcState*)(base + lay[0]);
    for (int ax = 0; ax < 3; ++ax) {
        a.pos[ax] = r.pos[ax];
        a.ast[ax] = r.st[ax];
    }
    a.qrange = r.qrange;
    a.key_lo = r.key_lo;
    a.key_hi = r.key_hi;
    a.ka = (unsigned long long*)(base + lay[1]);
    a.kb = (unsigned long long*)(base + lay[2]);
    a.va = (uint32_t*)(base + lay[3]);
    a.vb = (uint32_t*)(base + lay[4]);
    a.counts = (uint32_t*)(base + lay[5]);
    a.dbase = (unsigned long long*)(base + lay[6]);
    a.ntiles = (n + kTile - 1) / kTile;
    a.blk_first = (unsigned long long*)(base + lay[7]);
    a.blk_k = (uint32_t*)(base + lay[8]);
    a.blk_words = (unsigned long long*)(base + lay[9]);
    a.blk_exc = (unsigned long long*)(base + lay[10]);
    a.sub_off = (uint32_t*)(base + lay[11]);
    a.out = (uint8_t*)d_out;
    a.err = ctx->d_err;
    CpcState init;
    memset(&init, 0, sizeof(init));
    init.n = n;
    init.nb = (n + kCpcBlock - 1) / kCpcBlock;
    init.cap = out_cap;
    if (cudaMemcpyAsync(a.st, &init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    const int sms = sm_count_cpc();
    const uint32_t grid = (uint32_t)umin64((n + 255) / 256, (uint64_t)sms * 8u);
    cpc_params_kernel<<<1, 32, 0, s>>>(a);
    if (n) cpc_pairs_kernel<<<grid ? grid : 1, 256, 0, s>>>(a);
    // 8 passes of 8 bits; passes past the key width only copy
    unsigned long long *k0 = a.ka, *k1 = a.kb;
    uint32_t *v0 = a.va, *v1 = a.vb;
    for (uint32_t shift = 0; n && shift < 64; shift += 8) {
        a.shift = shift;
        cpc_hist_kernel<<<(uint32_t)a.ntiles, kSortT, 0, s>>>(a, k0);
        cpc_scan_tiles_kernel<<<kDigits, 1024, 0, s>>>(a);
        cpc_scan_digits_kernel<<<1, kDigits, 0, s>>>(a);
        cpc_scatter_kernel<<<(uint32_t)a.ntiles, kSortT, 0, s>>>(a, k0, v0, k1, v1);
        unsigned long long* tk = k0; k0 = k1; k1 = tk;
        uint32_t* tv = v0; v0 = v1; v1 = tv;
    }
    const uint64_t nb = (n + kCpcBlock - 1) / kCpcBlock;
    if (nb) cpc_block_kernel<<<(uint32_t)nb, kCpcThreads, 0, s>>>(a, k0, v0);
    cpc_layout_kernel<<<1, 1024, 0, s>>>(a);
    if (nb) cpc_pack_kernel<<<(uint32_t)nb, kCpcThreads, 0, s>>>(a, k0, v0);
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    if (perm_out && n &&
        cudaMemcpyAsync(perm_out, v0, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    return queue_result(ctx, &a.st->total, out_bytes, s);
}

}  // namespace szg

using namespace szg;

extern "C" {

size_t sz_cpc_max_bytes(size_t n) { return szg::cpc_max_bytes(n); }

sz_status sz_decompress_cpc(sz_ctx* ctx, const void* d_in, size_t in_bytes, float* const* d_out, size_t n_cap,
                            size_t* n_out, void* stream) {
    if (!ctx || !d_in || ((uintptr_t)d_in & 15u) || !d_out) return SZ_ERR_ARG;
    for (int ax = 0; ax < 3; ++ax)
        if ((n_cap && !d_out[ax]) || ((uintptr_t)d_out[ax] & 3u)) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t* base = nullptr;
    size_t lay[12];
    sz_status st = cpc_reserve(ctx, 0, &base, lay);
    if (st != SZ_OK) return st;
    CpcArgs a;
    memset(&a, 0, sizeof(a));
    a.st = (CpcState*)(base + lay[0]);
    a.in = (const uint8_t*)d_in;
    a.in_bytes = in_bytes;
    for (int ax = 0; ax < 3; ++ax) a.dst[ax] = d_out[ax];
    a.n_cap = n_cap;
    a.err = ctx->d_err;
    {
        ProfScope p(ctx, SZ_PHASE_DECODE, s);
        cpc_setup_kernel<<<1, 32, 0, s>>>(a);
        const int sms = sm_count_cpc();
        cpc_decode_kernel<<<sms * 4, 128, 0, s>>>(a);
        cpc_exceptions_kernel<<<sms, 256, 0, s>>>(a);
    }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return queue_result(ctx, &a.st->n, n_out, s);
}

}  // extern "C"
