// sz_encode.cuh -- a6 + a7: Huffman encoding of the codes into chunked
// sub-streams, the chunk tables and the escape records.
//
// A chunk of C elements is encoded by one block of NT = C / kRun threads;
// thread t holds the codeword-table entries of elements t*kRun .. t*kRun +
// kRun - 1 (entries: codeword << (32 - length) | escape << 5 | length, so a
// thread packs them as they stand).  One block scan gives each thread its
// start bit and escape index; each thread packs its codewords MSB-first into
// a zeroed shared buffer by funnel shifts (its first and last words, which it
// may share with its neighbours, by shared atomic OR; the words between by
// plain stores), and the chunk leaves with 128-bit stores.  Sub-stream k (G =
// C/64 elements) is threads [kG/kRun, (k+1)G/kRun), so its bit length is a
// shuffle reduction.  Escape records are rebuilt from global memory (rare).
// The chunk's word offset in the payload comes either
//   - from pass 1 of the two-pass encoder (encode_sizes_body): every chunk's
//     word count, scanned into the stream's chunk-word table with a look-back
//     over blocks instead of chunks; pass 2 (encode_pack_warp) then packs one
//     chunk per warp with no waits at all (arrays of 64 chunks or more), or
//   - from a decoupled look-back over the chunks before it, chunks being
//     taken in ticket order so that the look-back waits only on running
//     blocks (one pass: smaller arrays, the batched kernel's small arrays,
//     and codes recomputed from the input).
// Measured on GB300 (encode step of six 2^27-element arrays, rel eb 1e-4):
// one pass 2.18 ms; two passes 0.43 + 1.57 ms, 0.43 + 1.48 ms with the
// branch-free packing of pass 2 (1.63 with a branch per completed word), and
// 0.43 + 1.20 ms with sixteen codes per lane and round.
#pragma once
#include "sz_device.cuh"

namespace szg {

constexpr uint32_t kLookbackSpins = 1u << 22;

// Elements per thread of the stand-alone encode launches (chunks of up to
// 1024 * kEncRun elements use C / kEncRun threads; larger ones 1024).
// The launch bounds ask for kEncThreadsPerSM resident threads per SM.
// Measured on GB300 for 2^27-element arrays at C = 4096 (encode ms):
// run 16 / 1024 threads 0.50, run 32 / 512 0.51, run 16 / 768 0.57,
// run 8 / 1024 0.96; a shared-memory copy of the codeword table's hot
// window cost more in occupancy than it saved in gathers.
#ifndef SZ_ENC_RUN
#define SZ_ENC_RUN 16
#endif
#ifndef SZ_ENC_TPSM
#define SZ_ENC_TPSM 1024
#endif
constexpr int kEncRun = SZ_ENC_RUN;
constexpr int kEncThreadsPerSM = SZ_ENC_TPSM;
template <int C>
struct EncShape {
    static constexpr int kRun = (C / kEncRun > 1024) ? C / 1024 : kEncRun;
    static constexpr int kThreads = C / kRun;
    static constexpr int kMinBlocks = kThreads >= kEncThreadsPerSM ? 1 : kEncThreadsPerSM / kThreads;
};

// raw stream: words [wb, we) of the payload are the input bits (zero past n)
__device__ __forceinline__ void raw_copy_words(const CompressArgs& a, uint64_t wb, uint64_t we, uint64_t t0,
                                               uint64_t tstride) {
    if (a.st->total_bytes > a.out_cap) return;
    uint32_t* dst = reinterpret_cast<uint32_t*>(a.out + kHeaderBytes);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.in);
    for (uint64_t i = wb + t0; i < we; i += tstride) dst[i] = (i < a.n) ? __ldg(src + i) : 0u;
}

// dynamic shared memory of a persistent encoder for chunks of C elements:
// payload buffer (C words) and code stage (C / 2 words)
constexpr size_t enc_smem_bytes(int C) { return 4u * ((size_t)C + (size_t)C / 2); }

template <int NT>
struct EncSmem {
    unsigned long long ws64[NT / 32 + 1];
    unsigned long long prefix;
};

// The part of a chunk's encoding after each thread holds its kRun table
// entries r[j] (0 past the chunk's end): block scan of bit lengths and escape
// counts, packing, escape records, the chunk's word offset (LOOKBACK: by the
// look-back, after publishing the chunk's size; else from the chunk-word
// table of pass 1), the chunk tables and the coalesced copy of the payload.
// anchor (thread 0): the lattice value before the chunk; with LCF, anchor2 is
// the one before that and escapes carry the second difference.
template <int NT, int kRun, bool LCF = false, bool LOOKBACK = true>
__device__ __forceinline__ void encode_chunk_body(const CompressArgs& a, const LatticeParams& P, const uint32_t c,
                                                  const uint32_t (&r)[kRun], const long long anchor, uint32_t* buf,
                                                  EncSmem<NT>& esm, const long long anchor2 = 0) {
    constexpr int C = NT * kRun;
    unsigned long long& s_prefix = esm.prefix;
    ArrayState* st = a.st;
    const int tid = threadIdx.x;
    const uint64_t n = a.n, base = (uint64_t)c * C;
    const uint32_t cnt = (uint32_t)umin64(C, n - base);
    const float* in = a.in;
    const uint32_t e0 = tid * kRun;
    (void)cnt;
    uint32_t bits = 0, escs = 0;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
        bits += r[j] & 31u;
        escs += (r[j] >> 5) & 1u;
    }
    // one block scan of (escapes << 32 | bits)
    unsigned long long tot;
    const unsigned long long ex =
        block_exclusive_scan<NT>(((unsigned long long)escs << 32) | bits, esm.ws64, &tot);
    const uint32_t start = (uint32_t)ex, eoff = (uint32_t)(ex >> 32);
    const uint32_t chunk_bits = (uint32_t)tot;
    const uint32_t chunk_words = ((chunk_bits + 127u) >> 7) << 2;
    // sub-stream bit length: reduce over the G/32 lanes that share sub-stream
    constexpr int kLanesPerSub = C / kSubPerChunk / kRun;   // 1, 2, 4 or 8
    uint32_t sub_bits = bits;
#pragma unroll
    for (int o = 1; o < kLanesPerSub; o <<= 1) sub_bits += __shfl_xor_sync(0xffffffffu, sub_bits, o);

    // ---- publish this chunk's size for the look-back of later chunks --------------
    unsigned long long* status = a.chunk_status;
    constexpr unsigned long long FLAG_AGG = kLbAgg, FLAG_INC = kLbInc, FLAG_ERR = kLbErr;
    if (LOOKBACK && tid == 0) st_status(&status[c], (c == 0 ? FLAG_INC : FLAG_AGG) | chunk_words);
    // zero the payload area (the code entries are in registers now)
    for (uint32_t w4 = tid; w4 < chunk_words / 4; w4 += NT) reinterpret_cast<uint4*>(buf)[w4] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();

    // ---- pack into shared memory ----------------------------------------------------
    // cur holds the word being filled (fill bits used, from the top); a
    // codeword t (left-justified) adds t >> fill, and what does not fit is
    // the next word's start, t << (32 - fill) (a funnel shift: 0 when fill = 0).
    // A thread's first and last words may be shared with its neighbours
    // (atomic OR); the words in between are its own (plain stores).
    {
        uint32_t word = start >> 5, fill = start & 31u, cur = 0u;
        bool first = true;
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
            const uint32_t t = r[j] & ~255u;
            cur |= t >> fill;
            const uint32_t nxt = __funnelshift_r(0u, t, fill);
            fill += r[j] & 31u;
            if (fill >= 32u) {
                if (first) atomicOr(&buf[word], cur);
                else buf[word] = cur;
                first = false;
                ++word;
                cur = nxt;
                fill -= 32u;
            }
        }
        if (fill) atomicOr(&buf[word], cur);
    }

    // ---- escape records (rare): rebuilt from global memory ---------------------
    uint8_t* out = a.out;
    const uint64_t off_payload = st->off[S_PAYLOAD];
    const bool tables_ok = off_payload <= a.out_cap;
    if (escs && tables_ok) {
        uint8_t* esc_base = out + st->off[S_ESC] + (uint64_t)kEscBytes * (a.chunk_esc[c] + eoff);
        uint32_t idx = 0;
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
            if (r[j] & 32u) {
                uint64_t i = base + e0 + j;
                float x = __ldg(in + i);
                long long q, qp = 0, qpp = 0;
                bool vb, vv;
                lattice_q(x, P, q, vb);
                if (i > 0) lattice_q(__ldg(in + i - 1), P, qp, vv);
                if (LCF && i > 1) lattice_q(__ldg(in + i - 2), P, qpp, vv);
                uint8_t* rec = esc_base + (uint64_t)kEscBytes * idx++;
                *reinterpret_cast<long long*>(rec) = LCF ? (q - qp) - (qp - qpp) : q - qp;
                *reinterpret_cast<uint32_t*>(rec + 8) = vb ? __float_as_uint(x) : 0u;
                *reinterpret_cast<uint32_t*>(rec + 12) = vb ? 1u : 0u;
            }
        }
    }

    // ---- the chunk's word offset ------------------------------------------------------
    if (!LOOKBACK) {
        if (tid == 0) s_prefix = tables_ok ? reinterpret_cast<const uint64_t*>(out + st->off[S_CWORD])[c] : ~0ull;
    } else if (tid < 32 && c > 0) {
        // decoupled look-back, one warp, 32 predecessors per step
        unsigned long long excl = 0;
        const bool ok = lookback_prefix(status, c, kLookbackSpins, &excl);
        if (tid == 0) {
            if (!ok) {
                raise_err(a.err, E_TIMEOUT);
                st_status(&status[c], FLAG_ERR);
            } else {
                st_status(&status[c], FLAG_INC | (excl + chunk_words));
            }
            s_prefix = ok ? excl : ~0ull;
        }
    } else if (tid == 0) {
        s_prefix = 0ull;
    }
    __syncthreads();
    const unsigned long long prefix = s_prefix;
    if (prefix == ~0ull) return;

    // ---- tables ------------------------------------------------------------------
    const uint64_t chunk_end = off_payload + 4ull * (prefix + chunk_words);
    if (tables_ok) {
        if ((tid % kLanesPerSub) == 0) {
            const uint32_t k = tid / kLanesPerSub;
            reinterpret_cast<uint16_t*>(out + st->off[S_SUBLEN])[(uint64_t)c * kSubPerChunk + k] =
                (uint16_t)(e0 < cnt ? sub_bits : 0u);
        }
        if (tid == 0) {
            if (LOOKBACK) reinterpret_cast<uint64_t*>(out + st->off[S_CWORD])[c] = prefix;
            long long* anchors = reinterpret_cast<long long*>(out + st->off[S_ANCHOR]);
            if (LCF) {
                anchors[2 * (uint64_t)c] = anchor;
                anchors[2 * (uint64_t)c + 1] = anchor2;
            } else {
                anchors[c] = anchor;
            }
            if (LOOKBACK && c == a.n_chunks - 1)
                reinterpret_cast<uint64_t*>(out + st->off[S_CWORD])[c + 1] = prefix + chunk_words;
        }
    }
    if (LOOKBACK && c == a.n_chunks - 1 && tid == 0) {
        st->total_bytes = chunk_end;
        if (a.out_cap >= kHeaderBytes) {
            *reinterpret_cast<uint64_t*>(out + H_PWORDS) = prefix + chunk_words;
            *reinterpret_cast<uint64_t*>(out + H_TOTAL) = chunk_end;
        }
        if (chunk_end > a.out_cap) raise_err(a.err, E_CAPACITY);
    }
    if (tables_ok && chunk_end <= a.out_cap) {
        uint4* dst = reinterpret_cast<uint4*>(out + off_payload + 4ull * prefix);
        const uint4* src = reinterpret_cast<const uint4*>(buf);
        for (uint32_t w4 = tid; w4 < chunk_words / 4; w4 += NT) dst[w4] = src[w4];
    }
}

// Encode chunk c of array a with a block of NT threads, kRun = C / NT
// consecutive elements per thread.  buf: C words of shared memory.
template <int NT, int kRun, bool FROM_CODES>
__device__ void encode_chunk(const CompressArgs& a, const uint32_t c, uint32_t* buf, EncSmem<NT>& esm) {
    constexpr int C = NT * kRun;
    constexpr int kRunShift = kRun == 8 ? 3 : (kRun == 16 ? 4 : 5);
    static_assert(kRun == 8 || kRun == 16 || kRun == 32, "run length");
    ArrayState* st = a.st;
    const int tid = threadIdx.x, lane = tid & 31;
    const LatticeParams P = st->P;
    const uint64_t n = a.n, base = (uint64_t)c * C;
    const uint32_t cnt = (uint32_t)umin64(C, n - base);
    const float* in = a.in;
    const bool vec = ((uintptr_t)in & 15u) == 0;
    const uint32_t* enc = a.enc;
    const uint32_t e0 = tid * kRun;
    uint32_t r[kRun];
    long long anchor = 0;

    if (FROM_CODES) {
        // ---- pass 1+2: the quantizer's codes for elements e0 .. e0+31 ----------------
        const uint16_t* cp = a.codes + base + e0;
        uint32_t w[kRun / 2];
        if (e0 + kRun <= cnt) {
#pragma unroll
            for (int m = 0; m < kRun / 8; ++m) {
                uint4 v = __ldg(reinterpret_cast<const uint4*>(cp) + m);
                w[4 * m] = v.x; w[4 * m + 1] = v.y; w[4 * m + 2] = v.z; w[4 * m + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kRun / 2; ++j) {
                uint32_t lo = (e0 + 2 * j < cnt) ? __ldg(cp + 2 * j) : 0u;
                uint32_t hi = (e0 + 2 * j + 1 < cnt) ? __ldg(cp + 2 * j + 1) : 0u;
                w[j] = lo | (hi << 16);
            }
        }
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
            const uint32_t code = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu);
            r[j] = (e0 + j < cnt) ? __ldg(enc + code) : 0u;
        }
        if (tid == 0 && base > 0) {
            bool vv;
            lattice_q(__ldg(in + base - 1), P, anchor, vv);
        }
    } else {
    // ---- pass 1: codes and (codeword, length), coalesced -----------------------
#pragma unroll 2
    for (uint32_t e = 4 * tid; e < (uint32_t)C; e += 4 * NT) {
        float x[4];
        if (vec && e + 3 < cnt) {
            float4 v = __ldg(reinterpret_cast<const float4*>(in + base + e));
            x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = (e + j < cnt) ? __ldg(in + base + e + j) : 0.0f;
        }
        long long q[4];
        bool vb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], vb[j]);
        long long qprev = __shfl_up_sync(0xffffffffu, q[3], 1);
        if (lane == 0) {
            qprev = 0;
            if (base + e > 0 && e < cnt) {
                bool vv;
                lattice_q(__ldg(in + base + e - 1), P, qprev, vv);
            }
            if (e == 0) anchor = qprev;
        }
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pk[j] = 0u;
            if (e + j < cnt) {
                uint32_t code = make_code(q[j], j == 0 ? qprev : q[j - 1], vb[j]);
                pk[j] = __ldg(enc + code);
            }
        }
        *reinterpret_cast<uint4*>(&buf[swz(e, kRunShift)]) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    __syncthreads();

    // ---- pass 2: this thread's 32 consecutive entries ---------------------------
#pragma unroll
    for (int m = 0; m < kRun / 4; ++m) {
        uint4 v = *reinterpret_cast<const uint4*>(&buf[swz(e0 + 4 * m, kRunShift)]);
        r[4 * m] = v.x; r[4 * m + 1] = v.y; r[4 * m + 2] = v.z; r[4 * m + 3] = v.w;
    }
    }  // !FROM_CODES
    encode_chunk_body<NT, kRun>(a, P, c, r, anchor, buf, esm);
}

// Persistent, pipelined encoding of one array from the quantizer's codes
// (block of NT = C / kRun threads).  smem: C words (payload buffer) | C / 2
// words (code stage).  The block takes
// chunk tickets in order; while it encodes chunk c, the codes and the
// preceding element of its next ticket are already on their way into the
// stage (cp.async).  A block holds at most two tickets, and the smallest
// unfinished ticket is always being encoded, so the look-back still only
// waits on chunks that make progress.  s_prev: the element before the chunk
// (and, with LCF, the one before that in s_prev[1]).
template <int C, int NT, bool LCF = false, bool LOOKBACK = true>
__device__ __forceinline__ void encode_array_pipelined(const CompressArgs& a, uint32_t* smem, EncSmem<NT>& esm,
                                                       uint32_t* s_ticket, float* s_prev) {
    constexpr int kRun = C / NT;
    ArrayState* st = a.st;
    const int tid = threadIdx.x;
    uint32_t* buf = smem;
    uint16_t* stage = reinterpret_cast<uint16_t*>(smem + C);
    const LatticeParams P = st->P;
    const uint32_t s_stage = (uint32_t)__cvta_generic_to_shared(stage);
    const uint32_t s_prevp = (uint32_t)__cvta_generic_to_shared(s_prev);
    auto issue = [&](uint32_t cc) {
        // the chunk's C codes (the code buffer holds whole chunks) and, for thread 0,
        // the element before the chunk
        const uint16_t* src = a.codes + (uint64_t)cc * C;
        for (int i = tid; i < C / 8; i += NT)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s_stage + 16u * i),
                         "l"(__cvta_generic_to_global(src + 8 * i))
                         : "memory");
        if (tid == 0 && cc > 0)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s_prevp),
                         "l"(__cvta_generic_to_global(a.in + (uint64_t)cc * C - 1))
                         : "memory");
        if (LCF && tid == 0 && cc > 0)     // cc * C >= 2048, so the element two back exists
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s_prevp + 4u),
                         "l"(__cvta_generic_to_global(a.in + (uint64_t)cc * C - 2))
                         : "memory");
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (tid == 0) s_ticket[0] = atomicAdd(&st->ticket, 1u);
    __syncthreads();
    uint32_t c = s_ticket[0];
    if (c < a.n_chunks) issue(c);
    while (c < a.n_chunks) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();          // stage holds chunk c; buf is free
        const uint32_t cnt = (uint32_t)umin64(C, a.n - (uint64_t)c * C);
        const uint32_t e0 = tid * kRun;
        uint32_t w[kRun / 2];
#pragma unroll
        for (int m = 0; m < kRun / 8; ++m) {
            const uint4 v = *reinterpret_cast<const uint4*>(stage + e0 + 8 * m);
            w[4 * m] = v.x; w[4 * m + 1] = v.y; w[4 * m + 2] = v.z; w[4 * m + 3] = v.w;
        }
        // the next ticket's atomic is in flight while the codewords are looked up
        if (tid == 0) s_ticket[1] = atomicAdd(&st->ticket, 1u);
        long long anchor = 0, anchor2 = 0;
        if (tid == 0 && c > 0) {
            bool vv;
            lattice_q(s_prev[0], P, anchor, vv);
            if (LCF) lattice_q(s_prev[1], P, anchor2, vv);
        }
        uint32_t r[kRun];
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
            const uint32_t code = (j & 1) ? (w[j >> 1] >> 16) : (w[j >> 1] & 0xffffu);
            r[j] = (e0 + j < cnt) ? __ldg(a.enc + code) : 0u;
        }
        __syncthreads();          // the stage is read; the next ticket is known
        const uint32_t cn = s_ticket[1];
        if (cn < a.n_chunks) issue(cn);
        encode_chunk_body<NT, kRun, LCF, LOOKBACK>(a, P, c, r, anchor, buf, esm, anchor2);
        c = cn;
    }
}

// ---- two-pass encoding, pass 1 --------------------------------------------------------
// The word count of every chunk (its codes' lengths summed, padded to 128
// bits) and their exclusive scan: the stream's chunk-word table.  A block
// takes the next range of chunks by ticket (range t of nblocks: chunks
// [t nc / nblocks, (t + 1) nc / nblocks)), so it waits only on blocks that
// took their tickets earlier and are running: it sums its range one chunk per
// warp, publishes the range's total in the status word of its ticket, looks
// back over the earlier tickets for its prefix, and turns its range's counts
// into offsets.  The block of the last ticket writes the table's end, the
// header's payload size and total, and the stream size.  Reads the stored
// codes (the code buffer holds whole chunks).
constexpr int kSizeThreads = 256;

// codes kSizeWinLo .. kSizeWinLo + kSizeWin - 1 (deltas within +-kSizeWin / 2):
// their lengths are kept in shared memory by pass 1, one byte each.  Measured
// on GB300 (six 2^27-element arrays, rel eb 1e-4): pass 1 0.57 ms with every
// length read from the global table, 0.43 ms with this window.
constexpr uint32_t kSizeWin = 16384;
constexpr uint32_t kSizeWinLo = (uint32_t)kRadius - kSizeWin / 2;

struct EncSizesSmem {
    unsigned long long wsum[kSizeThreads / 32];
    unsigned long long ws64[kSizeThreads / 32 + 1];
    unsigned long long prefix, total;
    uint32_t ticket;
    uint8_t len[kSizeWin];
};

__device__ __forceinline__ uint32_t code_len(const uint32_t* enc, const uint8_t* win, uint32_t code) {
    const uint32_t w = code - kSizeWinLo;
    if (w < kSizeWin) return win[w];
    return __ldg(enc + code) & 31u;
}

// summed lengths of the eight codes in q (entries of codes past cnt, counted
// from the group's first element e, excluded)
__device__ __forceinline__ uint32_t code_bits8(const uint4 q, const uint32_t* enc, const uint8_t* win, uint32_t e,
                                               uint32_t cnt) {
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
    uint32_t bits = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t lo = code_len(enc, win, w[m] & 0xffffu), hi = code_len(enc, win, w[m] >> 16);
        bits += (e + 2 * m < cnt ? lo : 0u) + (e + 2 * m + 1 < cnt ? hi : 0u);
    }
    return bits;
}

template <int C>
__device__ void encode_sizes_body(const CompressArgs& a, uint32_t nblocks, EncSizesSmem& sm) {
    ArrayState* st = a.st;
    if (st->raw || a.n == 0) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nc = a.n_chunks;
    if (nblocks > nc) nblocks = nc;
    if (tid == 0) sm.ticket = atomicAdd(&st->size_ticket, 1u);
    for (uint32_t i = tid; i < kSizeWin; i += kSizeThreads) sm.len[i] = (uint8_t)(__ldg(a.enc + kSizeWinLo + i) & 31u);
    __syncthreads();
    const uint32_t t = sm.ticket;
    if (t >= nblocks) return;
    const uint32_t c0 = (uint32_t)((uint64_t)t * nc / nblocks), c1 = (uint32_t)((uint64_t)(t + 1) * nc / nblocks);
    const uint64_t off_payload = st->off[S_PAYLOAD];
    const bool tables_ok = off_payload <= a.out_cap;
    uint64_t* cword = reinterpret_cast<uint64_t*>(a.out + st->off[S_CWORD]);
    // ---- the range's chunks: words of each, one warp per chunk ---------------------
    unsigned long long wacc = 0;
    for (uint32_t c = c0 + warp; c < c1; c += kSizeThreads / 32) {
        const uint64_t base = (uint64_t)c * C;
        const uint32_t cnt = (uint32_t)umin64(C, a.n - base);
        const uint4* cp = reinterpret_cast<const uint4*>(a.codes + base);
        uint32_t bits = 0;
        // eight 16-byte loads in flight per lane, then their 64 independent lookups
        for (uint32_t v0 = lane; v0 < (uint32_t)C / 8; v0 += 256) {
            uint4 qq[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t v = v0 + 32u * u;
                qq[u] = v < (uint32_t)C / 8 ? __ldg(cp + v) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t v = v0 + 32u * u;
                if (v < (uint32_t)C / 8) bits += code_bits8(qq[u], a.enc, sm.len, 8 * v, cnt);
            }
        }
        bits = warp_reduce_sum(bits);
        const uint32_t words = ((bits + 127u) >> 7) << 2;
        if (lane == 0 && tables_ok) cword[c] = words;
        wacc += words;
    }
    if (lane == 0) sm.wsum[warp] = wacc;
    __syncthreads();
    // ---- the range's total, published; the prefix by the look-back over blocks ------
    if (warp == 0) {
        unsigned long long tot = lane < kSizeThreads / 32 ? sm.wsum[lane] : 0ull;
        tot = warp_reduce_sum(tot);
        unsigned long long* status = a.chunk_status;
        if (lane == 0) st_status(&status[t], (t == 0 ? kLbInc : kLbAgg) | tot);
        unsigned long long excl = 0;
        const bool ok = t == 0 || lookback_prefix(status, t, kLookbackSpins, &excl);
        if (lane == 0) {
            if (!ok) {
                raise_err(a.err, E_TIMEOUT);
                st_status(&status[t], kLbErr);
            } else if (t > 0) {
                st_status(&status[t], kLbInc | (excl + tot));
            }
            sm.prefix = ok ? excl : ~0ull;
            sm.total = tot;
        }
    }
    __syncthreads();
    const unsigned long long prefix = sm.prefix;
    if (prefix == ~0ull) return;
    // ---- counts -> offsets over the range, kSizeThreads chunks at a time -------------
    if (tables_ok) {
        unsigned long long run = prefix;
        for (uint32_t c = c0; c < c1; c += kSizeThreads) {
            const uint32_t ci = c + tid;
            const unsigned long long w = ci < c1 ? cword[ci] : 0ull;
            unsigned long long tot2;
            const unsigned long long ex = block_exclusive_scan<kSizeThreads>(w, sm.ws64, &tot2);
            if (ci < c1) cword[ci] = run + ex;
            run += tot2;
        }
    }
    if (t == nblocks - 1 && tid == 0) {
        const uint64_t pw = prefix + sm.total;
        const uint64_t end = off_payload + 4ull * pw;
        st->total_bytes = end;
        if (a.out_cap >= kHeaderBytes) {
            *reinterpret_cast<uint64_t*>(a.out + H_PWORDS) = pw;
            *reinterpret_cast<uint64_t*>(a.out + H_TOTAL) = end;
        }
        if (tables_ok) cword[nc] = pw;
        if (end > a.out_cap) raise_err(a.err, E_CAPACITY);
    }
}

// ---- two-pass encoding, pass 2: one warp per chunk ------------------------------------
// A warp takes a chunk by ticket and packs it in rounds of 512 codes, lane l
// holding codes 16l .. 16l+15 of the round: two 16-byte loads of codes (the
// next round's are in flight meanwhile), sixteen table lookups, one warp scan of
// (escapes, bits) for the lane's bit offset, funnel-shift packing into the
// warp's zeroed round buffer in shared memory (each completed word OR-ed in by
// a predicated shared reduction, so the lanes never diverge: a lane's first
// and last words may be shared with its neighbours).  Escapes are counted
// only in lanes that have one.  The round's complete words then leave with
// coalesced 32-bit
// stores, and its last, partial word opens the next round's buffer.  The
// chunk's payload offset comes from pass 1; the chunk ends with its partial
// word and zero padding to 128 bits.  Warps never wait for one another.
constexpr int kPackWarps = 8;
// dynamic shared memory of a packing block: the warps' round buffers
constexpr size_t pack_smem_bytes();
// three blocks per SM (80 registers; measured against 2 and 4 on GB300: two
// blocks of 94 registers pack six 2^27 arrays in 1.86 ms against 1.43 at rel
// eb 1e-4)
constexpr int kPackMinBlocks = 3;
// Codes per lane and round.  Measured on GB300 (six 2^27 arrays, rel eb 1e-3 /
// 1e-4 / 1e-5, packing pass): 16 codes 1.11 / 1.20 / 2.33 ms, 8 codes 1.36 /
// 1.43 / 2.39 ms (the round's scan, sub-stream sums, buffer clearing and
// copy-out are paid per round); 32 codes spill 312 bytes per thread.
#ifndef SZ_PACK_K
#define SZ_PACK_K 16
#endif
constexpr int kPackK = SZ_PACK_K;
static_assert(kPackK == 8 || kPackK == 16, "codes per lane");
// K codes x 32 lanes x 24 bits = 24 K words, plus the carried word
constexpr uint32_t kRoundBufWords = 32u * kPackK;
constexpr size_t pack_smem_bytes() { return 4u * (size_t)kPackWarps * kRoundBufWords; }
static_assert(kRoundBufWords >= 24u * kPackK + 2u, "a round's words and the carried one fit the buffer");

template <int C, bool LCF>
__device__ void encode_pack_warp(const CompressArgs& a, uint32_t* rbuf) {
    constexpr int G = C / kSubPerChunk;
    constexpr int K = kPackK, RS = 32 * K;   // codes per lane, per round
    constexpr int L = G / K;                 // lanes per sub-stream
    static_assert(L >= 1 && L <= 32, "sub-stream width");
    ArrayState* st = a.st;
    if (st->raw || a.n == 0) return;
    const int lane = threadIdx.x & 31;
    const uint64_t off_payload = st->off[S_PAYLOAD];
    if (off_payload > a.out_cap) return;     // no room for the tables (pass 1 reported the size)
    const LatticeParams P = st->P;
    uint8_t* out = a.out;
    const uint64_t* cword = reinterpret_cast<const uint64_t*>(out + st->off[S_CWORD]);
    uint16_t* sublen = reinterpret_cast<uint16_t*>(out + st->off[S_SUBLEN]);
    long long* anchors = reinterpret_cast<long long*>(out + st->off[S_ANCHOR]);
    uint32_t* payload = reinterpret_cast<uint32_t*>(out + off_payload);
    uint8_t* esc_out = out + st->off[S_ESC];
    const float* in = a.in;
    for (;;) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&st->ticket, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= a.n_chunks) return;
        const uint64_t base = (uint64_t)c * C;
        const uint32_t cnt = (uint32_t)umin64(C, a.n - base);
        const uint64_t wbeg = cword[c], wend = cword[c + 1];
        if (off_payload + 4ull * wend > a.out_cap) continue;     // does not fit (reported by pass 1)
        if (lane == 0) {
            long long q1 = 0, q2 = 0;
            bool vv;
            if (base > 0) lattice_q(__ldg(in + base - 1), P, q1, vv);
            if (LCF) {
                if (base > 1) lattice_q(__ldg(in + base - 2), P, q2, vv);
                anchors[2 * (uint64_t)c] = q1;
                anchors[2 * (uint64_t)c + 1] = q2;
            } else {
                anchors[c] = q1;
            }
        }
        const uint4* cp = reinterpret_cast<const uint4*>(a.codes + base);
        uint4 q4[K / 8];
#pragma unroll
        for (int i = 0; i < K / 8; ++i) q4[i] = __ldg(cp + (K / 8) * lane + i);
        uint32_t carry = 0u, carry_bits = 0u;
        uint64_t wout = wbeg;
        uint64_t esc_run = a.chunk_esc[c];
#pragma unroll 1
        for (uint32_t r = 0; r < (uint32_t)C / RS; ++r) {
            uint32_t w[K / 2];
#pragma unroll
            for (int i = 0; i < K / 8; ++i) {
                w[4 * i] = q4[i].x; w[4 * i + 1] = q4[i].y; w[4 * i + 2] = q4[i].z; w[4 * i + 3] = q4[i].w;
            }
            if (r + 1 < (uint32_t)C / RS) {
#pragma unroll
                for (int i = 0; i < K / 8; ++i) q4[i] = __ldg(cp + (RS / 8) * (r + 1) + (K / 8) * lane + i);
            }
            const uint32_t e0 = (uint32_t)RS * r + (uint32_t)K * lane;
            uint32_t ent[K];
            uint32_t bits = 0, escs = 0;
            if ((r + 1u) * (uint32_t)RS <= cnt) {        // a full round (the warp agrees)
#pragma unroll
                for (int j = 0; j < K; ++j) ent[j] = __ldg(a.enc + ((w[j >> 1] >> ((j & 1) * 16)) & 0xffffu));
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    ent[j] = (e0 + j < cnt) ? __ldg(a.enc + ((w[j >> 1] >> ((j & 1) * 16)) & 0xffffu)) : 0u;
            }
            uint32_t any = 0u;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                bits += ent[j] & 31u;
                any |= ent[j];
            }
            uint32_t emask = 0u;                  // the lane's escapes, bit j for code j
            if (any & 32u) {                      // escapes are rare: count them only where there are some
#pragma unroll
                for (int j = 0; j < K; ++j) emask |= ((ent[j] >> 5) & 1u) << j;
                escs = __popc(emask);
            }
            // warp scan of (escapes << 16 | bits): at most 32 K escapes and 768 K bits a round
            const uint32_t v = (escs << 16) | bits;
            uint32_t inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += t;
            }
            const uint32_t ex = inc - v, tot = __shfl_sync(0xffffffffu, inc, 31);
            // sub-stream bit lengths: lanes of one sub-stream reduce their bits
            uint32_t sb = bits;
#pragma unroll
            for (int o = 1; o < L; o <<= 1) sb += __shfl_xor_sync(0xffffffffu, sb, o);
            if ((lane & (L - 1)) == 0) sublen[(uint64_t)c * kSubPerChunk + e0 / G] = (uint16_t)(e0 < cnt ? sb : 0u);
            // the round buffer: the carried partial word, then zeros
            for (uint32_t i = lane; i < kRoundBufWords / 4; i += 32)
                reinterpret_cast<uint4*>(rbuf)[i] = make_uint4(i == 0 ? carry : 0u, 0u, 0u, 0u);
            __syncwarp();
            {
                // every completed word is OR-ed in by a predicated reduction:
                // no branch, so the lanes never diverge
                const uint32_t pos = carry_bits + (ex & 0xffffu);
                uint32_t addr = (uint32_t)__cvta_generic_to_shared(rbuf) + 4u * (pos >> 5), fill = pos & 31u, cw = 0u;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const uint32_t t = ent[j] & ~255u;
                    cw |= t >> fill;
                    const uint32_t nxt = __funnelshift_r(0u, t, fill);
                    fill += ent[j] & 31u;
                    const uint32_t done = fill >= 32u ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p red.shared.or.b32 [%0], %1;\n}" ::"r"(addr),
                                 "r"(cw), "r"(done)
                                 : "memory");
                    addr += 4u * done;
                    cw = done ? nxt : cw;
                    fill -= 32u * done;
                }
                asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %2, 0;\n @p red.shared.or.b32 [%0], %1;\n}" ::"r"(addr),
                             "r"(cw), "r"(fill)
                             : "memory");
            }
            // escape records (rare): rebuilt from the input
            if (emask) {
                uint64_t idx = esc_run + (ex >> 16);
                // by position bits, so that the entries stay in registers
                for (uint32_t mk = emask; mk; mk &= mk - 1u) {
                    const uint64_t i = base + e0 + (uint32_t)(__ffs(mk) - 1);
                    const float x = __ldg(in + i);
                    long long q, qp = 0, qpp = 0;
                    bool vb, vv;
                    lattice_q(x, P, q, vb);
                    if (i > 0) lattice_q(__ldg(in + i - 1), P, qp, vv);
                    if (LCF && i > 1) lattice_q(__ldg(in + i - 2), P, qpp, vv);
                    uint8_t* rec = esc_out + (uint64_t)kEscBytes * idx++;
                    *reinterpret_cast<long long*>(rec) = LCF ? (q - qp) - (qp - qpp) : q - qp;
                    *reinterpret_cast<uint32_t*>(rec + 8) = vb ? __float_as_uint(x) : 0u;
                    *reinterpret_cast<uint32_t*>(rec + 12) = vb ? 1u : 0u;
                }
            }
            esc_run += tot >> 16;
            __syncwarp();
            // the round's complete words out; the partial one carries over
            const uint32_t total = carry_bits + (tot & 0xffffu);
            const uint32_t nfull = total >> 5;
            for (uint32_t i = lane; i < nfull; i += 32) payload[wout + i] = rbuf[i];
            carry = rbuf[nfull];
            carry_bits = total & 31u;
            wout += nfull;
            __syncwarp();
        }
        // the last partial word and the zero padding to the chunk's end
        for (uint64_t i = wout + lane; i < wend; i += 32) payload[i] = i == wout ? carry : 0u;
    }
}

}  // namespace szg
