// k_decode.cu -- a9-a11: decompression.
//
// decode_setup (one block): validates the header against in_bytes, rebuilds
// the canonical code from the (symbol, length) list -- first code, count and
// base per length, left-justified limits, symbols in (length, symbol) order --
// and fills the lookup tables: a 12-bit first level (sym << 8 | len, or, for
// a prefix of longer codes, the shortest length under it << 8) and a second
// level over up to kLut2Max 16-bit prefixes past the first level's codes
// (codes of 13..16 bits, or the shortest longer length).  A code neither
// resolves is found by a short walk up the limits from that shortest length.
// In a stream of 64-symbol sub-streams the escape symbol's entries carry
// kEscMark instead of 0 (see decode_run16).  It also records the stream's
// largest chunk payload.
//
// decode (one persistent block per SM, split into up to twelve independent
// 64-thread "chunk teams", each with its own named barrier and mbarrier): a
// team takes one chunk at a time.  One thread stages the chunk's payload in
// shared memory with a single 1-D bulk copy and asks L2 to prefetch the team's
// next chunk; a block runs as many teams as leave each a stage that holds the
// stream's largest chunk (a chunk larger even for one team is read from
// global memory).  Thread k decodes sub-stream k (G symbols) from its start
// bit (team scan of the sub-stream bit lengths) into a row of 16-bit symbols,
// one table load per symbol and, in a staged full sub-stream, one refill of
// the 64-bit bit window per two symbols.  A team scan of the per-thread delta sums plus
// the chunk anchor gives each thread its starting lattice value (a10: the
// block-wide prefix scan; the anchor replaces the device-wide part).  Each
// thread then rebuilds its values x' = RN32(q*D) (a11) -- in 32-bit integers
// when no escape occurs and |q| provably stays within 2^24 -- a quarter of its
// run at a time into the now free stage, from which the team stores the
// quarter chunk with 128-bit coalesced stores.  Every table entry and payload
// word is bounds-checked against in_bytes; a bad stream sets E_CORRUPT.
// Streams with the LCF predictor (second differences, two anchors per chunk)
// take the same layout plus a second team scan for the entry state of each
// sub-stream, and rebuild in 32-bit integers only where a bound proves it
// exact, in non-inlined functions of their own.
#include "sz_blocksort.cuh"

namespace szg {

constexpr int kSetupThreads = 1024;
// The escape symbol as the lookup tables give it in streams of 64-symbol
// sub-streams: its low 16 bits (0) mark the escape in the symbol rows, and a
// sub-stream's sum of symbols counts the escapes from bit 22 up, since 64
// symbols below 2^16 sum to less than 2^22.
constexpr uint32_t kEscMark = 1u << 22;
constexpr int kDecThreads = kSubPerChunk;    // 64 threads per team
#ifndef SZ_DEC_TEAMS
#define SZ_DEC_TEAMS 12
#endif
constexpr int kMaxTeams = SZ_DEC_TEAMS;
// team t synchronises on named barrier t + 1; a CTA has barriers 0..15
static_assert(kMaxTeams >= 1 && kMaxTeams <= 15, "one named barrier per team");
constexpr int kDecBlock = kMaxTeams * kDecThreads;
constexpr size_t kDecDynSmem = 224u * 1024u;         // both lookup tables (48 KB) + team regions

struct SetupSmem {
    RadixSmem rs;
    uint32_t cnt[kMaxLen + 2];
    uint32_t ok, m, maxw;
    unsigned long long kraft;
};

__device__ __forceinline__ uint64_t rd64(const uint8_t* p) { return *reinterpret_cast<const uint64_t*>(p); }
__device__ __forceinline__ uint32_t rd32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ bool shape_ok(uint32_t C, uint32_t G) {
    return (C == 2048 || C == 4096 || C == 8192 || C == 16384) && G * kSubPerChunk == C;
}

// Validation and tables of one stream, by one block of kSetupThreads threads.
__device__ __forceinline__ void decode_setup_body(const DecompressArgs& a, SetupSmem& sm) {
    const int tid = threadIdx.x;
    ArrayState* st = a.st;
    const uint8_t* in = a.in;
    if (tid == 0) {
        // status: 0 ok, E_CORRUPT, E_CAPACITY or E_UNSUPPORTED
        uint32_t status = 0;
        st->dec_ok = 0;
        st->n_out = 0;
        st->raw = 0;
        sm.m = 0;
        if (a.in_bytes < kHeaderBytes || rd32(in + H_MAGIC) != kMagic ||
            *reinterpret_cast<const uint16_t*>(in + H_VERSION) != kVersion ||
            *reinterpret_cast<const uint16_t*>(in + H_HDRBYTES) != kHeaderBytes) {
            status = E_CORRUPT;
        } else {
            const uint64_t n = rd64(in + H_N), total = rd64(in + H_TOTAL), pw = rd64(in + H_PWORDS);
            const uint32_t flags = rd32(in + H_FLAGS), C = rd32(in + H_C), G = rd32(in + H_G);
            const uint32_t pred = in[H_PRED];
            const uint64_t na = pred == kPredLCF ? 2 : 1;     // chunk anchors per chunk
            const uint64_t nc = rd64(in + H_NCHUNKS), m = rd64(in + H_NSYM), E = rd64(in + H_NESC);
            uint64_t off[8];
            for (int s = 0; s < 8; ++s) off[s] = rd64(in + H_OFF + 8 * s);
            if (total > a.in_bytes || total < kHeaderBytes || n >= (1ull << 32) ||
                (pred != kPredLV && pred != kPredLCF))
                status = E_CORRUPT;
            st->pred = pred;
            for (int s = 0; !status && s < 8; ++s)
                if (off[s] < kHeaderBytes || off[s] > total || (off[s] & 15u) || (s && off[s] < off[s - 1]))
                    status = E_CORRUPT;
            if (!status && (pw > (1ull << 40) || off[S_PAYLOAD] + 4 * pw > total)) status = E_CORRUPT;
            if (!status) {
                if (flags & kFlagRaw) {
                    if (pw < n) status = E_CORRUPT;
                    st->raw = 1;
                } else if (n > 0) {
                    if (!shape_ok(C, G)) status = E_UNSUPPORTED;
                    else if (nc != (n + C - 1) / C || m == 0 || m > 65536 ||
                             off[S_LENS] - off[S_SYMS] < 2 * m || off[S_CWORD] - off[S_LENS] < m ||
                             off[S_ANCHOR] - off[S_CWORD] < 8 * (nc + 1) || off[S_CESC] - off[S_ANCHOR] < 8 * na * nc ||
                             off[S_SUBLEN] - off[S_CESC] < 8 * (nc + 1) ||
                             off[S_ESC] - off[S_SUBLEN] < 2 * nc * kSubPerChunk ||
                             E > n || E > (off[S_PAYLOAD] - off[S_ESC]) / kEscBytes)
                        status = E_CORRUPT;
                    sm.m = (uint32_t)m;
                }
            }
            if (!status) {
                st->n_out = n;
                for (int s = 0; s < 8; ++s) st->off[s] = off[s];
                if (n > a.n_cap) status = E_CAPACITY;
            } else if (status != E_CORRUPT) {
                st->n_out = n;
            }
        }
        if (status) raise_err(a.err, status);
        sm.ok = (status == 0);
    }
    __syncthreads();
    if (!sm.ok) return;
    if (st->raw || st->n_out == 0) {
        if (tid == 0) st->dec_ok = 1;
        return;
    }

    // canonical tables
    const uint32_t m = sm.m;
    const uint16_t* syms = reinterpret_cast<const uint16_t*>(in + st->off[S_SYMS]);
    const uint8_t* lens = in + st->off[S_LENS];
    uint32_t* scr = a.cb_scratch;
    for (int l = tid; l < kMaxLen + 2; l += kSetupThreads) sm.cnt[l] = 0;
    if (tid == 0) {
        sm.kraft = 0;
        sm.maxw = 0;
    }
    __syncthreads();
    unsigned long long kr = 0;
    for (uint32_t k = tid; k < m; k += kSetupThreads) {
        uint32_t l = lens[k];
        if (l < 1 || l > (uint32_t)kMaxLen || (k > 0 && syms[k] <= syms[k - 1])) { sm.ok = 0; l = 1; }
        atomicAdd(&sm.cnt[l], 1u);
        kr += 1ull << (kMaxLen - l);
        scr[k] = l;
        scr[65536 + k] = syms[k];
    }
    kr = warp_reduce_sum(kr);
    if ((tid & 31) == 0) atomicAdd(&sm.kraft, kr);
    __syncthreads();
    if (!sm.ok || sm.kraft > (1ull << kMaxLen)) {
        if (tid == 0) raise_err(a.err, E_CORRUPT);
        return;
    }
    uint32_t *kl = scr, *vl = scr + 65536;
    if (radix_pass<kSetupThreads>(scr, scr + 65536, scr + 2 * 65536, scr + 3 * 65536, m, 0, sm.rs)) {
        kl = scr + 2 * 65536;
        vl = scr + 3 * 65536;
    }
    if (tid == 0) {
        uint32_t c = 0, b = 0;
        sm.cnt[0] = 0;
        st->first[0] = st->count[0] = st->base[0] = st->lim[0] = 0;
        for (int l = 1; l <= kMaxLen; ++l) {
            c = (c + sm.cnt[l - 1]) << 1;
            st->first[l] = c;
            st->count[l] = sm.cnt[l];
            st->base[l] = b;
            st->lim[l] = (c + sm.cnt[l]) << (kMaxLen - l);
            b += sm.cnt[l];
        }
        st->lim[kMaxLen + 1] = 0xffffffffu;
    }
    __syncthreads();
    // First level: 12-bit prefixes.  Codes of up to 12 bits fill their
    // prefixes with sym << 8 | len; every prefix of longer codes holds the
    // shortest length under it, lmin << 8 (len field 0; lmin 25 = no code).
    // Second level: the 16-bit prefixes from lim[12] on, at most kLut2Max of
    // them -- codes of 13..16 bits as sym << 8 | len, prefixes of longer
    // codes as lmin << 8.  lmin(x) = the first l with x < lim[l], because the
    // codes of length l occupy [lim[l-1], lim[l]) in left-justified order.
    constexpr int kSh = kMaxLen - kLut2Bits;
    const uint32_t l2_lo = st->lim[kLutBits] >> kSh;
    const uint32_t l2_n = umin32(kLut2Max, 65536u - l2_lo);
    const uint32_t l2_short = (st->lim[kLut2Bits] >> kSh) - l2_lo;   // entries of codes <= 16 bits
    uint32_t* lut2 = a.lut + (1u << kLutBits);
    const uint32_t p1_lo = st->lim[kLutBits] >> (kMaxLen - kLutBits);
    for (uint32_t i = tid; i < (1u << kLutBits); i += kSetupThreads) {
        uint32_t v = 0u;
        if (i >= p1_lo) {
            uint32_t l = kLutBits + 1;
            while (l <= (uint32_t)kMaxLen && (i << (kMaxLen - kLutBits)) >= st->lim[l]) ++l;
            v = l << 8;
        }
        a.lut[i] = v;
    }
    for (uint32_t i = tid; i < l2_n; i += kSetupThreads) {
        uint32_t v = 0u;
        if (i >= l2_short) {
            uint32_t l = kLut2Bits + 1;
            while (l <= (uint32_t)kMaxLen && ((l2_lo + i) << kSh) >= st->lim[l]) ++l;
            v = l << 8;
        }
        lut2[i] = v;
    }
    __syncthreads();
    const uint32_t esc_sym = rd32(in + H_G) == 64u ? kEscMark : 0u;   // the header is valid here
    for (uint32_t p = tid; p < m; p += kSetupThreads) {
        uint32_t l = kl[p], s = vl[p];
        a.by_len[p] = (uint16_t)s;
        const uint32_t code = st->first[l] + (p - st->base[l]);
        if (s == 0u) s = esc_sym;
        if (l <= (uint32_t)kLutBits) {
            uint32_t lo = code << (kLutBits - l), hi = (code + 1) << (kLutBits - l);
            for (uint32_t e = lo; e < hi; ++e) a.lut[e] = (s << 8) | l;
        } else if (l <= (uint32_t)kLut2Bits) {
            uint32_t lo = (code << (kLut2Bits - l)) - l2_lo, hi = ((code + 1) << (kLut2Bits - l)) - l2_lo;
            for (uint32_t e = lo; e < hi && e < l2_n; ++e) lut2[e] = (s << 8) | l;
        }
    }
    // the largest chunk payload, which sets how many teams a block runs (the
    // stage of each must hold it); malformed offsets count as empty chunks here
    // and are rejected where the chunk is decoded
    {
        const uint64_t* cw = reinterpret_cast<const uint64_t*>(in + st->off[S_CWORD]);
        const uint64_t nc = rd64(in + H_NCHUNKS);
        uint32_t mx = 0;
        for (uint64_t c = tid; c < nc; c += kSetupThreads) {
            const uint64_t wb = cw[c], we = cw[c + 1];
            if (we > wb) mx = max(mx, (uint32_t)umin64(we - wb, 1u << 24));
        }
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) atomicMax(&sm.maxw, mx);
    }
    __syncthreads();
    if (tid == 0) {
        st->l2_lo = l2_lo;
        st->l2_n = l2_n;
        st->max_cw = sm.maxw;
        st->dec_ok = 1;
    }
}

__global__ void __launch_bounds__(kSetupThreads) decode_setup_kernel(DecompressArgs a) {
    __shared__ SetupSmem sm;
    decode_setup_body(a, sm);
}

// Bit reader over a chunk payload in shared or global memory.  Two 32-bit
// words (hi, lo) hold the stream from word pos-2 on; the next codeword starts
// b bits into hi.  peek() returns the 32 bits from there by one funnel shift;
// consume() advances and pulls in one word when b passes 32 (predicated, so
// lanes do not diverge).  Words at or past `end` read as zero, so a bad
// stream cannot make it read outside the chunk: PAD = false tests the index
// and loads only when a word is due; PAD = true (a staged chunk, whose stage
// holds a zero word at `end`) loads every step from the index clamped to
// `end`, which costs fewer instructions than the test.
template <bool PAD>
struct BitReaderT {
    const uint32_t* words;
    uint32_t pos, end, hi, lo, b;
    __device__ __forceinline__ void init(const uint32_t* w, uint32_t begin_bit, uint32_t end_word) {
        words = w;
        end = end_word;
        const uint32_t p = begin_bit >> 5;
        hi = p < end ? w[p] : 0u;
        lo = p + 1 < end ? w[p + 1] : 0u;
        pos = p + 2;
        b = begin_bit & 31u;
    }
    static constexpr bool kPad = PAD;
    __device__ __forceinline__ uint32_t peek() const { return __funnelshift_l(lo, hi, b); }
    // the window from bit b for b up to 48 (at least 16 valid bits)
    __device__ __forceinline__ uint32_t peek16() const {
        const bool past = b >= 32u;
        return __funnelshift_l(past ? 0u : lo, past ? lo : hi, b);
    }
    __device__ __forceinline__ void advance(uint32_t len) { b += len; }
    __device__ __forceinline__ void consume(uint32_t len) {
        b += len;
        refill();
    }
    __device__ __forceinline__ void refill() {
        const bool need = b >= 32u;
        const uint32_t nxt = PAD ? words[umin32(pos, end)] : ((need && pos < end) ? words[pos] : 0u);
        hi = need ? lo : hi;
        lo = need ? nxt : lo;
        pos += need ? 1u : 0u;
        b -= need ? 32u : 0u;
    }
    __device__ __forceinline__ uint32_t bit_pos() const { return (pos - 2u) * 32u + b; }
};

// Team-level primitives: a team is 64 threads (2 warps) with named barrier
// id team + 1.
__device__ __forceinline__ void team_sync(int team) {
    asm volatile("bar.sync %0, %1;" :: "r"(team + 1), "r"(kDecThreads) : "memory");
}

template <typename T>
__device__ __forceinline__ T team_exclusive_scan(T v, T* ws, int team, int k, T* total) {
    T inc = warp_inclusive_scan(v);
    if ((k & 31) == 31) ws[k >> 5] = inc;
    team_sync(team);
    T w0 = ws[0];
    T r = inc - v + ((k >> 5) ? w0 : T(0));
    *total = w0 + ws[1];
    team_sync(team);
    return r;
}
// The same without the closing barrier: for a buffer the team writes next
// only after a later team barrier (each scan of a chunk has its own buffer).
template <typename T>
__device__ __forceinline__ T team_exclusive_scan_once(T v, T* ws, int team, int k, T* total) {
    T inc = warp_inclusive_scan(v);
    if ((k & 31) == 31) ws[k >> 5] = inc;
    team_sync(team);
    T w0 = ws[0];
    T r = inc - v + ((k >> 5) ? w0 : T(0));
    *total = w0 + ws[1];
    return r;
}

struct DecSmem {
    uint32_t lim[kMaxLen + 2];            // left-justified (24-bit) end of each length's codes
    uint32_t first[kMaxLen + 2], base[kMaxLen + 2];
    uint32_t ws32[kMaxTeams][2], ws32b[kMaxTeams][2];
    long long ws64[kMaxTeams][2];
    unsigned long long mbar[kMaxTeams];   // each team's payload barrier
    uint32_t mph[kMaxTeams];              // its current phase parity
};

// polls of a team's payload barrier before the copy counts as lost
constexpr uint32_t kStageSpins = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One arrival (the thread that issues the copy) plus the copy's bytes complete
// a phase of a team's payload barrier.  The caller synchronises the block
// before a team stages.
__device__ __forceinline__ void init_stage_barriers(DecSmem& sm, int tid) {
    if (tid < kMaxTeams) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[tid])) : "memory");
        sm.mph[tid] = 0u;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < kStageSpins; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// A chunk's payload (words: a multiple of 4, 16-byte aligned in global and
// shared memory alike, as every chunk is padded to 128 bits) into the team's
// stage: one thread issues a single 1-D bulk copy that completes on the team's
// barrier, and the team waits for the barrier's phase.  The caller
// team-synchronises afterwards and then calls stage_done.  Returns false
// (E_TIMEOUT raised) if the copy never landed; the team then waits once more,
// bounded, for it before giving up.
__device__ __forceinline__ bool stage_chunk(const uint32_t* src, uint32_t* stage, uint32_t words, DecSmem& sm,
                                            int team, int k, uint32_t* err) {
    const uint32_t bar = smem_u32(&sm.mbar[team]);
    const uint32_t ph = sm.mph[team];
    if (k == 0) {
        const uint32_t bytes = 4u * words;
        // the team's earlier generic accesses to the stage come before the copy's writes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        if (bytes)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(stage)),
                "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(bar)
                : "memory");
    }
    if (mbar_wait(bar, ph)) return true;
    if (k == 0) raise_err(err, E_TIMEOUT);
    mbar_wait(bar, ph);
    return false;
}

// After the team barrier that follows stage_chunk: the next copy waits on the
// barrier's other phase.
__device__ __forceinline__ void stage_done(DecSmem& sm, int team, int k) {
    if (k == 0) sm.mph[team] ^= 1u;
}

// dynamic shared memory: the lookup tables (the 12-bit first level, then the
// second level's window, as the codebook lays them out in global memory),
// then one region per team
constexpr uint32_t kTabWords = (1u << kLutBits) + kLut2Max;
constexpr size_t kTabBytes = sizeof(uint32_t) * kTabWords;
constexpr uint32_t kRegionPool = (uint32_t)((kDecDynSmem - kTabBytes) / 4);   // words for the team regions

// Teams per block for chunks of C elements whose largest payload is max_cw
// words: the most (up to kMaxTeams) whose region -- the symbol or value slots
// and the stage -- still stages the largest chunk; a stream with chunks larger
// even for one team reads those from global memory.
// LV streams keep the symbols as 16-bit words (C / 2 words) and need a stage
// of at least C / 4 words, which carries the values out; LCF streams keep C
// 32-bit slots.
__device__ __forceinline__ int teams_for(uint32_t C, uint32_t max_cw, bool lcf) {
    (void)lcf;   // LV and LCF streams alike keep 16-bit symbol rows
    const uint32_t need = C / 2u + umax32(max_cw, C / 4u) + 4u;
    int t = kMaxTeams;
    while (t > 1 && ((kRegionPool / (uint32_t)t) & ~3u) < need) --t;
    return t;
}

// A code longer than the second level covers: walk the left-justified limits
// from `len` (the shortest length under the code's prefix).  Returns
// sym << 8 | len, or 0 for a window that starts no code (len is never 0).
__device__ __noinline__ uint32_t decode_long(uint32_t w24, uint32_t len, const DecSmem& sm, const uint16_t* by_len) {
    while (len <= (uint32_t)kMaxLen && w24 >= sm.lim[len]) ++len;
    if (len > (uint32_t)kMaxLen) return 0u;
    return ((uint32_t)by_len[sm.base[len] + (w24 >> (kMaxLen - len)) - sm.first[len]] << 8) | len;
}

// One symbol, one table load: a window whose 16-bit prefix falls in the
// second level's range (which starts where the codes of up to 12 bits end)
// reads the second level, any other the first; both resolve codes of up to
// 16 bits and mark longer ones with the shortest length under the prefix, for
// the walk.  MARK: the stream's tables give the escape as kEscMark, and so
// does the walk.
template <bool MARK, class BR>
__device__ __forceinline__ uint32_t decode_symbol(BR& br, const DecSmem& sm, const uint32_t* tab, uint32_t l2_lo,
                                                  uint32_t l2_n, const uint16_t* by_len, bool& bad) {
    const uint32_t w = br.peek();
    const uint32_t i2 = (w >> (32 - kLut2Bits)) - l2_lo;   // wraps above l2_n below the range
    uint32_t ent = tab[i2 < l2_n ? (1u << kLutBits) + i2 : (w >> (32 - kLutBits))];
    if ((ent & 255u) == 0u) {
        ent = decode_long(w >> (32 - kMaxLen), ent >> 8, sm, by_len);
        bad = bad || ent == 0u;
        if (MARK && ent != 0u && (ent >> 8) == 0u) ent |= kEscMark << 8;
    }
    br.consume(ent & 255u);
    return ent >> 8;
}

// Two symbols with one refill: after a code of at most 16 bits the 64-bit
// window still holds the 16 bits the tables read; a longer code (the walk)
// refills before the next symbol, and the walk itself reads a refilled window.
template <bool MARK, class BR>
__device__ __forceinline__ void decode_pair(BR& br, const DecSmem& sm, const uint32_t* tab, uint32_t l2_lo,
                                            uint32_t l2_n, const uint16_t* by_len, uint32_t& s0, uint32_t& s1,
                                            bool& bad) {
    uint32_t w = br.peek();
    uint32_t i2 = (w >> (32 - kLut2Bits)) - l2_lo;
    uint32_t ent = tab[i2 < l2_n ? (1u << kLutBits) + i2 : (w >> (32 - kLutBits))];
    if ((ent & 255u) == 0u) {
        ent = decode_long(w >> (32 - kMaxLen), ent >> 8, sm, by_len);
        bad = bad || ent == 0u;
        if (MARK && ent != 0u && (ent >> 8) == 0u) ent |= kEscMark << 8;
        br.consume(ent & 255u);
    } else {
        br.advance(ent & 255u);
    }
    s0 = ent >> 8;
    w = br.peek16();
    i2 = (w >> (32 - kLut2Bits)) - l2_lo;
    ent = tab[i2 < l2_n ? (1u << kLutBits) + i2 : (w >> (32 - kLutBits))];
    if ((ent & 255u) == 0u) {
        br.refill();
        w = br.peek();
        ent = decode_long(w >> (32 - kMaxLen), ent >> 8, sm, by_len);
        bad = bad || ent == 0u;
        if (MARK && ent != 0u && (ent >> 8) == 0u) ent |= kEscMark << 8;
    }
    br.consume(ent & 255u);
    s1 = ent >> 8;
}

// The LV path's 16-bit symbol rows: row k (sub-stream k) holds G symbols as
// G / 4 units of 8 bytes; unit u sits at u ^ (k / max(1, 16 / NU)) mod NU, so
// the 16 rows a half-warp writes or reads at one unit index hit distinct banks.
// (sh = log2(max(1, 16 / NU)), precomputed per stream)
__device__ __forceinline__ uint32_t sym_unit(uint32_t u, uint32_t k, uint32_t NU, uint32_t sh) {
    return u ^ ((k >> sh) & (NU - 1u));
}
// The value rows of a round: row k holds F 16-byte groups; group m sits at
// m ^ (k / max(1, 8 / F)) mod F, free of conflicts for the row writes and for
// the copy-out's reads alike.
// (sh = log2(max(1, 8 / F)))
__device__ __forceinline__ uint32_t val_unit(uint32_t m, uint32_t row, uint32_t F, uint32_t sh) {
    return m ^ ((row >> sh) & (F - 1u));
}

// Phase 1 of one sub-stream: nsym symbols into the thread's 16-bit row.
// Returns their sum and adds their escapes to nesc: counted one by one, or
// (MARK) read from bits 22 and up of the sum of the marked symbols.
template <bool FULL, bool MARK, class BR>
__device__ __forceinline__ uint32_t decode_run16(BR& br, const DecSmem& sm, const uint32_t* tab, uint32_t l2_lo,
                                                 uint32_t l2_n, const uint16_t* by_len, uint2* srow, uint32_t NU,
                                                 uint32_t ush, uint32_t k, uint32_t nsym, uint32_t& nesc, bool& bad) {
    uint32_t ssum = 0;
    for (uint32_t j4 = 0; j4 < nsym; j4 += 4) {
        uint32_t s[4] = {0u, 0u, 0u, 0u};
        if constexpr (FULL && BR::kPad) {
            decode_pair<MARK>(br, sm, tab, l2_lo, l2_n, by_len, s[0], s[1], bad);
            decode_pair<MARK>(br, sm, tab, l2_lo, l2_n, by_len, s[2], s[3], bad);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ssum += s[t];
                if (!MARK) nesc += (s[t] == 0u);
            }
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (FULL || j4 + t < nsym) {
                    s[t] = decode_symbol<MARK>(br, sm, tab, l2_lo, l2_n, by_len, bad);
                    ssum += s[t];
                    if (!MARK) nesc += (s[t] == 0u);
                }
            }
        }
        // the low halves: a marked escape stores as 0
        srow[sym_unit(j4 >> 2, k, NU, ush)] = make_uint2(__byte_perm(s[0], s[1], 0x5410), __byte_perm(s[2], s[3], 0x5410));
    }
    if (MARK) {
        nesc += ssum >> 22;
        ssum &= kEscMark - 1u;
    }
    return ssum;
}

// Per-stream decode parameters, read from the validated header and state.
struct DecArray {
    const uint64_t* cword;
    const long long* anchor;
    const uint64_t* cesc;
    const uint16_t* sublen;
    const uint8_t* escs;
    const uint32_t* payload;
    const uint16_t* by_len;
    float* out;
    uint64_t n, nc, E, pw;
    uint32_t C, G, gshift, l2_lo, l2_n, max_cw;
    float D;
    bool vec;
    bool lcf;          // second-difference (LCF) stream: two anchors per chunk
};

__device__ __forceinline__ void dec_array(const DecompressArgs& a, DecArray& d) {
    const ArrayState* st = a.st;
    const uint8_t* in = a.in;
    d.n = st->n_out;
    d.out = a.out;
    d.vec = ((uintptr_t)a.out & 15u) == 0;
    d.payload = reinterpret_cast<const uint32_t*>(in + st->off[S_PAYLOAD]);
    if (st->raw) return;
    d.C = rd32(in + H_C);
    d.G = rd32(in + H_G);
    d.gshift = 31 - __clz(d.G);
    d.nc = rd64(in + H_NCHUNKS);
    d.E = rd64(in + H_NESC);
    d.pw = rd64(in + H_PWORDS);
    d.D = __uint_as_float(rd32(in + H_D));
    d.cword = reinterpret_cast<const uint64_t*>(in + st->off[S_CWORD]);
    d.anchor = reinterpret_cast<const long long*>(in + st->off[S_ANCHOR]);
    d.cesc = reinterpret_cast<const uint64_t*>(in + st->off[S_CESC]);
    d.sublen = reinterpret_cast<const uint16_t*>(in + st->off[S_SUBLEN]);
    d.escs = in + st->off[S_ESC];
    d.by_len = a.by_len;
    d.l2_lo = st->l2_lo;
    d.l2_n = st->l2_n;
    d.max_cw = st->max_cw;
    d.lcf = st->pred == kPredLCF;
}

// Block-wide: the stream's first- and second-level tables and limits into
// shared memory.
__device__ __forceinline__ void load_dec_tables(const DecompressArgs& a, const DecArray& d, DecSmem& sm,
                                                uint32_t* tab) {
    const int tid = threadIdx.x;
    const ArrayState* st = a.st;
    for (uint32_t i = tid; i < (1u << kLutBits) + d.l2_n; i += blockDim.x) tab[i] = __ldg(a.lut + i);
    if (tid < kMaxLen + 2) {
        sm.first[tid] = st->first[tid];
        sm.base[tid] = st->base[tid];
        sm.lim[tid] = st->lim[tid];
    }
}


// One LV chunk by one team through 16-bit symbol rows (sym16: C / 2 words)
// and the stage (stage_words >= C / 4): stage the payload (stage_chunk; a
// chunk larger than the stage is read from global memory), decode
// each sub-stream into its row, scan the escapes and the delta sums, then four
// rounds: each thread rebuilds G / 4 values into its row of the stage (free
// once the payload is decoded) and the team stores the quarter chunk with
// coalesced 16-byte stores.  next: the chunk this team takes next (L2
// prefetch), or >= nc.  Returns false (and raises E_CORRUPT) on a bad chunk.
// GT: the sub-stream length when known at compile time (64, i.e. C = 4096, the
// fixed rule for arrays above 2^16 elements), so that the row and swizzle
// arithmetic folds to constants; 0 takes it from the stream.
template <uint32_t GT>
__device__ __forceinline__ bool decode_chunk_lv16(const DecArray& d, DecSmem& sm, const uint32_t* tab,
                                                  uint32_t* sym16, uint32_t* stage, uint32_t stage_words, int team,
                                                  int k, uint64_t c, uint64_t next, uint32_t* err,
                                                  uint32_t* ctr = nullptr, uint32_t* slot = nullptr,
                                                  uint32_t* next_out = nullptr) {
    // ctr: the stream's unit counter; the team's next ticket is drawn here and
    // handed out through `slot` after the staging barrier (next_out), and it
    // is also the chunk whose payload is prefetched into L2
    if (ctr != nullptr && k == 0) {
        const uint32_t t = atomicAdd(ctr, 1u);
        *slot = t;
        next = t;
    }
    const uint32_t G = GT ? GT : d.G, C = GT ? GT * kSubPerChunk : d.C;
    const uint32_t NU = G / 4u, F = G / 16u, VR = G / 4u;
    const uint32_t gsh = GT ? (31u - __clz(GT)) : d.gshift;   // log2 G (5 .. 8)
    const uint32_t ush = gsh >= 6 ? 0u : 6u - gsh;       // log2 max(1, 16 / NU)
    const uint32_t vsh = gsh >= 7 ? 0u : 7u - gsh;       // log2 max(1, 8 / F)
    const uint64_t base = c * C;
    const uint32_t cnt = (uint32_t)umin64(C, d.n - base);
    const uint64_t wb = d.cword[c], we = d.cword[c + 1];
    const uint64_t eb = d.cesc[c], ee = d.cesc[c + 1];
    const bool hdr_bad = (wb > we || we > d.pw || eb > ee || ee > d.E || ((wb | we) & 3u));
    const uint32_t e0 = k * G;
    const uint32_t nsym = e0 < cnt ? umin32(G, cnt - e0) : 0u;
    const uint32_t sl = d.sublen[c * kSubPerChunk + k];
    uint32_t tot_bits;
    const uint32_t start = team_exclusive_scan_once<uint32_t>(sl, sm.ws32[team], team, k, &tot_bits);
    if (hdr_bad || (uint64_t)tot_bits > 32ull * (we - wb)) {
        if (k == 0) raise_err(err, E_CORRUPT);
        return false;
    }
    // ---- stage the chunk payload; prefetch the team's next chunk into L2 --------
    const uint32_t cw_words = (uint32_t)(we - wb);
    const bool staged = cw_words < stage_words;     // the stage holds the payload and a zero word after it
    if (staged && !stage_chunk(d.payload + wb, stage, cw_words, sm, team, k, err)) return false;
    if (staged && k == 0) stage[cw_words] = 0u;
    if (k == 0 && next < d.nc) {
        const uint64_t nb = d.cword[next], ne = d.cword[next + 1];
        if (nb < ne && ne <= d.pw && !(nb & 3u) && !(ne & 3u) && ne - nb < (1u << 24)) {
            const uint32_t* p = d.payload + nb;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)),
                         "r"((uint32_t)(4 * (ne - nb)))
                         : "memory");
        }
    }
    team_sync(team);
    if (staged) stage_done(sm, team, k);
    if (ctr != nullptr) *next_out = *slot;
    // ---- phase 1: the sub-stream's symbols into the thread's row -----------------
    uint2* srow = reinterpret_cast<uint2*>(sym16) + (size_t)k * NU;
    uint32_t nesc = 0, ssum, end_bit;
    bool bad = false;
    if (staged) {
        BitReaderT<true> br;
        br.init(stage, start, cw_words);
        ssum = nsym == G
                   ? decode_run16<true, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc, bad)
                   : decode_run16<false, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc,
                                                   bad);
        end_bit = br.bit_pos();
    } else {
        BitReaderT<false> br;
        br.init(d.payload + wb, start, cw_words);
        ssum = decode_run16<false, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc, bad);
        end_bit = br.bit_pos();
    }
    bad = bad || end_bit - start != sl;
    // ---- escapes and the team-wide prefix (the stage is free after these barriers) --
    uint32_t tot_esc;
    const uint32_t eoff =
        team_exclusive_scan_once<uint32_t>(nesc + (bad ? 0x10000u : 0u), sm.ws32b[team], team, k, &tot_esc);
    if ((tot_esc >> 16) || eb + tot_esc != ee) {
        if (k == 0) raise_err(err, E_CORRUPT);
        return false;
    }
    long long sum = (long long)ssum - (long long)kRadius * (long long)(nsym - nesc);
    for (uint32_t t = 0; t < nesc; ++t)
        sum += *reinterpret_cast<const long long*>(d.escs + (uint64_t)kEscBytes * (eb + eoff + t));
    long long tot_sum;
    const long long pre = team_exclusive_scan_once<long long>(sum, sm.ws64[team], team, k, &tot_sum);
    // ---- phase 2: four rounds of G / 4 values through the stage -------------------
    const float D = d.D;
    const long long q_fast = (1ll << 24) - (long long)G * (kRadius - 1);
    long long q = d.anchor[c] + pre;
    const bool fast = nesc == 0 && q >= -q_fast && q <= q_fast;
    uint64_t ecur = eb + eoff;
    float* dst = d.out + base;
    const bool full_vec = d.vec && cnt == C;
    float4* tr = reinterpret_cast<float4*>(stage);
    const uint32_t fsh = gsh - 4u;                       // log2 F
    for (uint32_t r = 0; r < 4; ++r) {
        if (fast) {
            // |q| stays within 2^24: exact in 32-bit integers and in one int -> float
            int qi = (int)q;
            for (uint32_t m = 0; m < F; ++m) {
                const uint2 u = srow[sym_unit(r * F + m, k, NU, ush)];
                qi += (int)(u.x & 0xffffu) - kRadius; const float v0 = __fmul_rn((float)qi, D);
                qi += (int)(u.x >> 16) - kRadius;     const float v1 = __fmul_rn((float)qi, D);
                qi += (int)(u.y & 0xffffu) - kRadius; const float v2 = __fmul_rn((float)qi, D);
                qi += (int)(u.y >> 16) - kRadius;     const float v3 = __fmul_rn((float)qi, D);
                tr[(k << fsh) + val_unit(m, k, F, vsh)] = make_float4(v0, v1, v2, v3);
            }
            q = qi;
        } else {
            for (uint32_t m = 0; m < F; ++m) {
                const uint2 u = srow[sym_unit(r * F + m, k, NU, ush)];
                const uint32_t sy[4] = {u.x & 0xffffu, u.x >> 16, u.y & 0xffffu, u.y >> 16};
                float v[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    v[t] = 0.0f;
                    if (r * VR + 4 * m + t < nsym) {
                        if (sy[t] != 0u) {
                            q += (long long)sy[t] - kRadius;
                            v[t] = recon_f(q, D);
                        } else {
                            const uint8_t* rec = d.escs + (uint64_t)kEscBytes * ecur++;
                            q += *reinterpret_cast<const long long*>(rec);
                            v[t] = (rd32(rec + 12) & 1u) ? __uint_as_float(rd32(rec + 8)) : recon_f(q, D);
                        }
                    }
                }
                tr[(k << fsh) + val_unit(m, k, F, vsh)] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        team_sync(team);
        for (uint32_t g = k; g < kDecThreads * F; g += kDecThreads) {
            const uint32_t row = g >> fsh, m = g & (F - 1u);
            const float4 val = tr[(row << fsh) + val_unit(m, row, F, vsh)];
            const uint32_t e = row * G + r * VR + 4 * m;
            if (full_vec) {
                *reinterpret_cast<float4*>(dst + e) = val;
            } else {
                const float vv[4] = {val.x, val.y, val.z, val.w};
                for (int j = 0; j < 4 && e + j < cnt; ++j) dst[e + j] = vv[j];
            }
        }
        team_sync(team);
    }
    return true;
}

// One LCF chunk by one team, in the layout of decode_chunk_lv16 (16-bit symbol
// rows, then four rounds of values through the stage).  With the first
// difference f_i = q_i - q_{i-1}: f_i = f_{i-1} + delta_i and q_i = q_{i-1} + f_i.
// A sub-stream of L deltas maps (f, q) to (f + S, q + L f + T), S the sum of its
// deltas and T the sum of their running sums; a team scan of S gives each
// sub-stream its entry f, a second one of L * (S-prefix) + T its entry q
// (unsigned arithmetic wraps like the two's-complement recurrence).  A
// sub-stream without escapes whose every partial q provably stays within 2^24
// (from the largest running sums of its deltas) rebuilds in 32-bit integers.
template <uint32_t GT>
__device__ __forceinline__ bool decode_chunk_lcf16(const DecArray& d, DecSmem& sm, const uint32_t* tab,
                                                   uint32_t* sym16, uint32_t* stage, uint32_t stage_words, int team,
                                                   int k, uint64_t c, uint64_t next, uint32_t* err) {
    const uint32_t G = GT ? GT : d.G, C = GT ? GT * kSubPerChunk : d.C;
    const uint32_t NU = G / 4u, F = G / 16u, VR = G / 4u;
    const uint32_t gsh = GT ? (31u - __clz(GT)) : d.gshift;   // log2 G (5 .. 8)
    const uint32_t ush = gsh >= 6 ? 0u : 6u - gsh;       // log2 max(1, 16 / NU)
    const uint32_t vsh = gsh >= 7 ? 0u : 7u - gsh;       // log2 max(1, 8 / F)
    const uint64_t base = c * C;
    const uint32_t cnt = (uint32_t)umin64(C, d.n - base);
    const uint64_t wb = d.cword[c], we = d.cword[c + 1];
    const uint64_t eb = d.cesc[c], ee = d.cesc[c + 1];
    const bool hdr_bad = (wb > we || we > d.pw || eb > ee || ee > d.E || ((wb | we) & 3u));
    const uint32_t e0 = k * G;
    const uint32_t nsym = e0 < cnt ? umin32(G, cnt - e0) : 0u;
    const uint32_t sl = d.sublen[c * kSubPerChunk + k];
    uint32_t tot_bits;
    const uint32_t start = team_exclusive_scan<uint32_t>(sl, sm.ws32[team], team, k, &tot_bits);
    if (hdr_bad || (uint64_t)tot_bits > 32ull * (we - wb)) {
        if (k == 0) raise_err(err, E_CORRUPT);
        return false;
    }
    // ---- stage the chunk payload; prefetch the team's next chunk into L2 --------
    const uint32_t cw_words = (uint32_t)(we - wb);
    const bool staged = cw_words < stage_words;     // the stage holds the payload and a zero word after it
    if (staged && !stage_chunk(d.payload + wb, stage, cw_words, sm, team, k, err)) return false;
    if (staged && k == 0) stage[cw_words] = 0u;
    if (k == 0 && next < d.nc) {
        const uint64_t nb = d.cword[next], ne = d.cword[next + 1];
        if (nb < ne && ne <= d.pw && !(nb & 3u) && !(ne & 3u) && ne - nb < (1u << 24)) {
            const uint32_t* p = d.payload + nb;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)),
                         "r"((uint32_t)(4 * (ne - nb)))
                         : "memory");
        }
    }
    team_sync(team);
    if (staged) stage_done(sm, team, k);
    // ---- phase 1: the sub-stream's symbols into the thread's row -----------------
    uint2* srow = reinterpret_cast<uint2*>(sym16) + (size_t)k * NU;
    uint32_t nesc = 0, ssum, end_bit;
    bool bad = false;
    if (staged) {
        BitReaderT<true> br;
        br.init(stage, start, cw_words);
        ssum = nsym == G
                   ? decode_run16<true, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc, bad)
                   : decode_run16<false, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc,
                                                   bad);
        end_bit = br.bit_pos();
    } else {
        BitReaderT<false> br;
        br.init(d.payload + wb, start, cw_words);
        ssum = decode_run16<false, GT == 64>(br, sm, tab, d.l2_lo, d.l2_n, d.by_len, srow, NU, ush, k, nsym, nesc, bad);
        end_bit = br.bit_pos();
    }
    bad = bad || end_bit - start != sl;
    // ---- escapes, S, and the entry f -------------------------------------------
    uint32_t tot_esc;
    const uint32_t eoff =
        team_exclusive_scan<uint32_t>(nesc + (bad ? 0x10000u : 0u), sm.ws32b[team], team, k, &tot_esc);
    if ((tot_esc >> 16) || eb + tot_esc != ee) {
        if (k == 0) raise_err(err, E_CORRUPT);
        return false;
    }
    long long S = (long long)ssum - (long long)kRadius * (long long)(nsym - nesc);
    for (uint32_t t = 0; t < nesc; ++t)
        S += *reinterpret_cast<const long long*>(d.escs + (uint64_t)kEscBytes * (eb + eoff + t));
    long long tot_s;
    const long long pre = team_exclusive_scan<long long>(S, sm.ws64[team], team, k, &tot_s);
    // ---- T and the largest running sums over the row ---------------------------
    uint64_t run = 0, T = 0, mr = 0, mt = 0;
    {
        uint64_t ec = eb + eoff;
        for (uint32_t j4 = 0; j4 < nsym; j4 += 4) {
            const uint2 u = srow[sym_unit(j4 >> 2, k, NU, ush)];
            const uint32_t sy[4] = {u.x & 0xffffu, u.x >> 16, u.y & 0xffffu, u.y >> 16};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (j4 + t < nsym) {
                    const uint64_t dl = sy[t] ? (uint64_t)((long long)sy[t] - kRadius)
                                              : *reinterpret_cast<const uint64_t*>(d.escs + (uint64_t)kEscBytes * ec++);
                    run += dl;
                    T += run;
                    mr = umax64(mr, (uint64_t)llabs((long long)run));
                    mt = umax64(mt, (uint64_t)llabs((long long)T));
                }
            }
        }
    }
    long long tot_t;
    const long long preT =
        team_exclusive_scan<long long>((long long)((uint64_t)nsym * (uint64_t)pre + T), sm.ws64[team], team, k, &tot_t);
    const uint64_t qm1 = (uint64_t)d.anchor[2 * c], qm2 = (uint64_t)d.anchor[2 * c + 1];
    const uint64_t f0 = qm1 - qm2;
    uint64_t f = f0 + (uint64_t)pre;
    uint64_t q = qm1 + (uint64_t)e0 * f0 + (uint64_t)preT;
    // every q of the row is q + (j + 1) f + (a partial T), every f is f + (a running sum)
    const uint64_t af = (uint64_t)llabs((long long)f), aq = (uint64_t)llabs((long long)q);
    const bool fast = nesc == 0 && af <= (1ull << 24) && mr <= (1ull << 24) && mt <= (1ull << 26) &&
                      aq + (uint64_t)nsym * af + mt <= (1ull << 24);
    // ---- phase 2: four rounds of G / 4 values through the stage -------------------
    const float D = d.D;
    uint64_t ecur = eb + eoff;
    float* dst = d.out + base;
    const bool full_vec = d.vec && cnt == C;
    float4* tr = reinterpret_cast<float4*>(stage);
    const uint32_t fsh = gsh - 4u;                       // log2 F
    for (uint32_t r = 0; r < 4; ++r) {
        if (fast) {
            // 32-bit, wrapping past the row's end (those values are not stored)
            uint32_t fu = (uint32_t)f, qu = (uint32_t)q;
            for (uint32_t m = 0; m < F; ++m) {
                const uint2 u = srow[sym_unit(r * F + m, k, NU, ush)];
                fu += (u.x & 0xffffu) - (uint32_t)kRadius; qu += fu; const float v0 = __fmul_rn((float)(int)qu, D);
                fu += (u.x >> 16) - (uint32_t)kRadius;     qu += fu; const float v1 = __fmul_rn((float)(int)qu, D);
                fu += (u.y & 0xffffu) - (uint32_t)kRadius; qu += fu; const float v2 = __fmul_rn((float)(int)qu, D);
                fu += (u.y >> 16) - (uint32_t)kRadius;     qu += fu; const float v3 = __fmul_rn((float)(int)qu, D);
                tr[(k << fsh) + val_unit(m, k, F, vsh)] = make_float4(v0, v1, v2, v3);
            }
            f = (uint64_t)(long long)(int)fu;
            q = (uint64_t)(long long)(int)qu;
        } else {
            for (uint32_t m = 0; m < F; ++m) {
                const uint2 u = srow[sym_unit(r * F + m, k, NU, ush)];
                const uint32_t sy[4] = {u.x & 0xffffu, u.x >> 16, u.y & 0xffffu, u.y >> 16};
                float v[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    v[t] = 0.0f;
                    if (r * VR + 4 * m + t < nsym) {
                        if (sy[t] != 0u) {
                            f += (uint64_t)((long long)sy[t] - kRadius);
                            q += f;
                            v[t] = recon_f((long long)q, D);
                        } else {
                            const uint8_t* rec = d.escs + (uint64_t)kEscBytes * ecur++;
                            f += *reinterpret_cast<const uint64_t*>(rec);
                            q += f;
                            v[t] = (rd32(rec + 12) & 1u) ? __uint_as_float(rd32(rec + 8)) : recon_f((long long)q, D);
                        }
                    }
                }
                tr[(k << fsh) + val_unit(m, k, F, vsh)] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        team_sync(team);
        for (uint32_t g = k; g < kDecThreads * F; g += kDecThreads) {
            const uint32_t row = g >> fsh, m = g & (F - 1u);
            const float4 val = tr[(row << fsh) + val_unit(m, row, F, vsh)];
            const uint32_t e = row * G + r * VR + 4 * m;
            if (full_vec) {
                *reinterpret_cast<float4*>(dst + e) = val;
            } else {
                const float vv[4] = {val.x, val.y, val.z, val.w};
                for (int j = 0; j < 4 && e + j < cnt; ++j) dst[e + j] = vv[j];
            }
        }
        team_sync(team);
    }
    return true;
}

// LCF streams run their team loops in separate, non-inlined functions, so the
// LV path the kernels inline keeps its own code and registers (the stream
// parameters are passed by value: a reference would pin the caller's copy in
// local memory).  Strided chunks (decode_kernel) and counted units
// (decode_multi_kernel, s_unit: the block's per-team unit slots).
__device__ __noinline__ void decode_team_lcf_strided(const DecArray d, DecSmem& sm, const uint32_t* tab,
                                                     uint32_t* xs, uint32_t stage_words, int team, int k,
                                                     uint64_t c0, uint64_t stride, uint32_t* err) {
    for (uint64_t c = c0; c < d.nc; c += stride)
        if (!(d.G == 64u ? decode_chunk_lcf16<64>(d, sm, tab, xs, xs + d.C / 2, stage_words, team, k, c, c + stride, err)
                         : decode_chunk_lcf16<0>(d, sm, tab, xs, xs + d.C / 2, stage_words, team, k, c, c + stride, err)))
            return;
}

__device__ __noinline__ void decode_team_lcf_counted(const DecArray d, DecSmem& sm, const uint32_t* tab,
                                                     uint32_t* xs, uint32_t stage_words, int team, int k,
                                                     uint32_t* ctr, uint32_t nu, uint32_t* s_unit, uint32_t* err) {
    if (k == 0) s_unit[team] = atomicAdd(ctr, 1u);
    team_sync(team);
    uint32_t u = s_unit[team];
    team_sync(team);
    while (u < nu) {
        if (k == 0) s_unit[team] = atomicAdd(ctr, 1u);      // the next ticket, prefetched while u decodes
        team_sync(team);
        const uint32_t un = s_unit[team];
        team_sync(team);
        const uint64_t nx = un < nu ? un : ~0ull;
        if (!(d.G == 64u ? decode_chunk_lcf16<64>(d, sm, tab, xs, xs + d.C / 2, stage_words, team, k, u, nx, err)
                         : decode_chunk_lcf16<0>(d, sm, tab, xs, xs + d.C / 2, stage_words, team, k, u, nx, err)))
            return;
        u = un;
    }
}

// team region of a block: `slots` words of symbol (or value) slots -- C / 2
// for LV streams' 16-bit rows, C for LCF -- then the payload stage
__device__ __forceinline__ uint32_t* team_region(uint4* dyn, int teams, int team, uint32_t* stage_words,
                                                 uint32_t slots) {
    const uint32_t region_words = (kRegionPool / teams) & ~3u;
    *stage_words = region_words - slots;  // multiple of 4
    return reinterpret_cast<uint32_t*>(dyn) + kTabWords + (size_t)team * region_words;
}

__global__ void __launch_bounds__(kDecBlock, 1) decode_kernel(DecompressArgs a) {
    __shared__ DecSmem sm;
    extern __shared__ uint4 dyn_smem[];
    const ArrayState* st = a.st;
    const int tid = threadIdx.x;
    if (!st->dec_ok) return;
    DecArray d;
    dec_array(a, d);
    if (d.n == 0) return;
    if (st->raw) {
        const uint32_t* src = d.payload;
        uint32_t* dst = reinterpret_cast<uint32_t*>(a.out);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < d.n; i += (uint64_t)gridDim.x * blockDim.x)
            dst[i] = __ldg(src + i);
        return;
    }
    uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);
    init_stage_barriers(sm, tid);
    load_dec_tables(a, d, sm, tab);
    __syncthreads();
    const int teams = teams_for(d.C, d.max_cw, d.lcf);
    const int team = tid / kDecThreads, k = tid % kDecThreads;
    if (team >= teams) return;
    uint32_t stage_words;
    const uint32_t slots = d.C / 2;
    uint32_t* xs = team_region(dyn_smem, teams, team, &stage_words, slots);
    const uint64_t stride = (uint64_t)gridDim.x * teams;
    if (d.lcf) {
        decode_team_lcf_strided(d, sm, tab, xs, stage_words, team, k, (uint64_t)blockIdx.x * teams + team, stride,
                                a.err);
        return;
    }
    for (uint64_t c = (uint64_t)blockIdx.x * teams + team; c < d.nc; c += stride)
        if (!(d.G == 64u
                  ? decode_chunk_lv16<64>(d, sm, tab, xs, xs + slots, stage_words, team, k, c, c + stride, a.err)
                  : decode_chunk_lv16<0>(d, sm, tab, xs, xs + slots, stage_words, team, k, c, c + stride, a.err)))
            return;
}

// ---- batched decompression ---------------------------------------------------
// setup: one block per stream; also writes the stream's decode units (chunks,
// or 4096-word pieces of a raw stream; 0 for a rejected stream)
constexpr uint32_t kRawUnit = 4096;

__global__ void __launch_bounds__(kSetupThreads) decode_setup_multi_kernel(const DecompressArgs* args,
                                                                           uint32_t* units, uint32_t* ctr) {
    __shared__ SetupSmem sm;
    __shared__ DecompressArgs sa;
    if (threadIdx.x == 0) sa = args[blockIdx.x];
    __syncthreads();
    decode_setup_body(sa, sm);
    __syncthreads();
    if (threadIdx.x == 0) {
        const ArrayState* st = sa.st;
        uint64_t u = 0;
        if (st->dec_ok && st->n_out) u = st->raw ? (st->n_out + kRawUnit - 1) / kRawUnit : rd64(sa.in + H_NCHUNKS);
        units[blockIdx.x] = (uint32_t)umin64(u, 0xffffffffu);
        ctr[blockIdx.x] = 0u;
    }
}

// exclusive prefix of the units over the k streams (one block)
__global__ void __launch_bounds__(1024) decode_units_scan_kernel(const uint32_t* units, uint64_t* uoff, uint32_t k) {
    __shared__ unsigned long long ws[33];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b = 0; b < k; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const unsigned long long v = i < k ? units[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_scan<1024>(v, ws, &tot);
        if (i < k) uoff[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) uoff[k] = carry;
}

// last index i < k with uoff[i] <= x (uoff non-decreasing)
__device__ __forceinline__ uint32_t find_stream(const uint64_t* uoff, uint32_t k, uint64_t x) {
    uint32_t lo = 0, hi = k;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (uoff[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// All streams' units in one launch, shared out dynamically: every stream has
// a unit counter (zeroed by the setup launch) from which teams take one chunk
// (or one raw piece) at a time.  Block b starts at the stream holding unit
// F b / B of the flattened list -- so blocks start spread in proportion to
// the work -- and sweeps the streams cyclically from there, visiting each
// once: it loads a stream's tables, its teams drain the stream's counter, and
// the block moves on.  Streams with fast and slow chunks thus end together.
// A team takes its next unit's ticket before decoding the current one and
// asks L2 to prefetch that unit's payload (a fixed distance ahead would miss:
// only the blocks on the same stream draw from its counter).  A bad chunk
// stops its team on that stream only.
__global__ void __launch_bounds__(kDecBlock, 1) decode_multi_kernel(const DecompressArgs* args, const uint64_t* uoff,
                                                                    uint32_t* ctr, uint32_t k) {
    __shared__ DecSmem sm;
    __shared__ DecompressArgs sa;
    __shared__ uint32_t s_go;
    __shared__ uint32_t s_unit[kMaxTeams];
    extern __shared__ uint4 dyn_smem[];
    const int tid = threadIdx.x;
    const uint64_t F = uoff[k];
    if (F == 0) return;
    init_stage_barriers(sm, tid);      // the stream loop's first block barrier publishes them
    uint32_t* tab = reinterpret_cast<uint32_t*>(dyn_smem);
    const int team = tid / kDecThreads, kk = tid % kDecThreads;
    uint32_t i = find_stream(uoff, k, F * blockIdx.x / gridDim.x);
    for (uint32_t v = 0; v < k; ++v, i = (i + 1 == k) ? 0 : i + 1) {
        const uint32_t nu = (uint32_t)(uoff[i + 1] - uoff[i]);
        if (nu == 0) continue;
        __syncthreads();          // the previous stream's teams are done with the tables
        if (tid == 0) {
            s_go = *reinterpret_cast<volatile const uint32_t*>(ctr + i) < nu;
            if (s_go) sa = args[i];
        }
        __syncthreads();
        if (!s_go) continue;
        DecArray d;
        dec_array(sa, d);
        const bool raw = sa.st->raw != 0;
        if (!raw) {
            load_dec_tables(sa, d, sm, tab);
            __syncthreads();
        }
        const int teams = raw ? kMaxTeams : teams_for(d.C, d.max_cw, d.lcf);
        if (team >= teams) continue;
        uint32_t stage_words = 0;
        const uint32_t slots = d.C / 2;
        uint32_t* xs = raw ? nullptr : team_region(dyn_smem, teams, team, &stage_words, slots);
        if (!raw && d.lcf) {
            decode_team_lcf_counted(d, sm, tab, xs, stage_words, team, kk, ctr + i, nu, s_unit, sa.err);
            continue;
        }
        // a team holds two tickets: while it decodes unit u, unit un (its next)
        // is prefetched into L2
        if (kk == 0) s_unit[team] = atomicAdd(ctr + i, 1u);
        team_sync(team);
        uint32_t u = s_unit[team];
        team_sync(team);
        while (u < nu) {
            if (!raw) {
                // the next ticket travels with the chunk's staging barrier
                uint32_t un = 0;
                if (!(d.G == 64u
                          ? decode_chunk_lv16<64>(d, sm, tab, xs, xs + slots, stage_words, team, kk, u, ~0ull, sa.err,
                                                  ctr + i, &s_unit[team], &un)
                          : decode_chunk_lv16<0>(d, sm, tab, xs, xs + slots, stage_words, team, kk, u, ~0ull, sa.err,
                                                 ctr + i, &s_unit[team], &un)))
                    break;
                u = un;
                continue;
            }
            // a raw stream: a 4096-word piece per unit
            if (kk == 0) s_unit[team] = atomicAdd(ctr + i, 1u);
            team_sync(team);
            const uint32_t un = s_unit[team];
            team_sync(team);
            uint32_t* dst = reinterpret_cast<uint32_t*>(sa.out);
            const uint64_t e1 = umin64(d.n, ((uint64_t)u + 1) * kRawUnit);
            for (uint64_t e = (uint64_t)u * kRawUnit + kk; e < e1; e += kDecThreads) dst[e] = __ldg(d.payload + e);
            u = un;
        }
    }
}

void launch_decode_setup(const DecompressArgs* a, int k, void* stream) {
    for (int i = 0; i < k; ++i) decode_setup_kernel<<<1, kSetupThreads, 0, (cudaStream_t)stream>>>(a[i]);
}

static int decode_grid() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
        cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecDynSmem);
        cudaFuncSetAttribute(decode_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDecDynSmem);
    }
    return sms;
}

void launch_decode(const DecompressArgs* a, int k, void* stream) {
    const int sms = decode_grid();
    for (int i = 0; i < k; ++i) {
        const int div = a[i].grid_div > 1 ? (int)a[i].grid_div : 1;
        const int grid = sms / div > 0 ? sms / div : 1;
        decode_kernel<<<grid, kDecBlock, kDecDynSmem, (cudaStream_t)stream>>>(a[i]);
    }
}

void launch_decode_multi_setup(const DecompressArgs* d_args, uint32_t k, uint32_t* d_units, uint64_t* d_uoff,
                               void* stream) {
    if (k == 0) return;
    cudaStream_t s = (cudaStream_t)stream;
    // the units words double as the per-stream unit counters after the scan
    decode_setup_multi_kernel<<<k, kSetupThreads, 0, s>>>(d_args, d_units, d_units + k);
    decode_units_scan_kernel<<<1, 1024, 0, s>>>(d_units, d_uoff, k);
}

void launch_decode_multi(const DecompressArgs* d_args, uint32_t k, uint32_t* d_units, const uint64_t* d_uoff,
                         void* stream) {
    if (k == 0) return;
    const int sms = decode_grid();
    decode_multi_kernel<<<sms, kDecBlock, kDecDynSmem, (cudaStream_t)stream>>>(d_args, d_uoff, d_units + k, k);
}

}  // namespace szg
