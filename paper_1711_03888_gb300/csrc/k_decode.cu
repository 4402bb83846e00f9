// k_decode.cu -- a9-a11: decompression.
//
// decode_setup (one block): validates the header against in_bytes, rebuilds
// the canonical code from the (symbol, length) list -- first code, count and
// base per length, symbols in (length, symbol) order -- and fills an 11-bit
// direct lookup table.
//
// decode (persistent 64-thread blocks, one chunk at a time): thread k decodes
// sub-stream k (G symbols) from its start bit (block scan of the sub-stream
// bit lengths), keeping the codes in a swizzled shared buffer and the sum of
// its deltas.  A block scan of the sums plus the chunk anchor gives every
// thread its starting lattice value (a10: block-wide prefix scan; the anchor
// replaces the device-wide part).  Each thread then rebuilds its values
// x' = RN32(q*D) (a11), escapes patch delta / raw bits, and the chunk leaves
// with 128-bit coalesced stores.  Every table entry and payload word is
// bounds-checked against in_bytes; a bad stream sets E_CORRUPT.
#include "sz_blocksort.cuh"

namespace szg {

constexpr int kSetupThreads = 1024;
constexpr int kDecThreads = kSubPerChunk;    // 64

struct SetupSmem {
    RadixSmem rs;
    uint32_t cnt[kMaxLen + 2];
    uint32_t ok, m;
    unsigned long long kraft;
};

__device__ __forceinline__ uint64_t rd64(const uint8_t* p) { return *reinterpret_cast<const uint64_t*>(p); }
__device__ __forceinline__ uint32_t rd32(const uint8_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

__global__ void __launch_bounds__(kSetupThreads) decode_setup_kernel(DecompressArgs a) {
    __shared__ SetupSmem sm;
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
            const uint64_t nc = rd64(in + H_NCHUNKS), m = rd64(in + H_NSYM), E = rd64(in + H_NESC);
            uint64_t off[8];
            for (int s = 0; s < 8; ++s) off[s] = rd64(in + H_OFF + 8 * s);
            if (total > a.in_bytes || total < kHeaderBytes || n >= (1ull << 32)) status = E_CORRUPT;
            for (int s = 0; !status && s < 8; ++s)
                if (off[s] < kHeaderBytes || off[s] > total || (off[s] & 15u) || (s && off[s] < off[s - 1]))
                    status = E_CORRUPT;
            if (!status && (pw > (1ull << 40) || off[S_PAYLOAD] + 4 * pw > total)) status = E_CORRUPT;
            if (!status) {
                if (flags & kFlagRaw) {
                    if (pw < n) status = E_CORRUPT;
                    st->raw = 1;
                } else if (n > 0) {
                    const bool shape = (C == 2048 || C == 4096 || C == 8192 || C == 16384) && G * kSubPerChunk == C;
                    if (!shape) status = E_UNSUPPORTED;
                    else if (nc != (n + C - 1) / C || m == 0 || m > 65536 ||
                             off[S_LENS] - off[S_SYMS] < 2 * m || off[S_CWORD] - off[S_LENS] < m ||
                             off[S_ANCHOR] - off[S_CWORD] < 8 * (nc + 1) || off[S_CESC] - off[S_ANCHOR] < 8 * nc ||
                             off[S_SUBLEN] - off[S_CESC] < 8 * (nc + 1) ||
                             off[S_ESC] - off[S_SUBLEN] < 2 * nc * kSubPerChunk ||
                             off[S_PAYLOAD] - off[S_ESC] < (uint64_t)kEscBytes * E)
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
    if (tid == 0) sm.kraft = 0;
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
        st->first[0] = st->count[0] = st->base[0] = 0;
        for (int l = 1; l <= kMaxLen; ++l) {
            c = (c + sm.cnt[l - 1]) << 1;
            st->first[l] = c;
            st->count[l] = sm.cnt[l];
            st->base[l] = b;
            b += sm.cnt[l];
        }
    }
    for (uint32_t i = tid; i < (1u << kLutBits); i += kSetupThreads) a.lut[i] = 0u;
    __syncthreads();
    for (uint32_t p = tid; p < m; p += kSetupThreads) {
        uint32_t l = kl[p], s = vl[p];
        a.by_len[p] = (uint16_t)s;
        if (l <= (uint32_t)kLutBits) {
            uint32_t code = st->first[l] + (p - st->base[l]);
            uint32_t lo = code << (kLutBits - l), hi = (code + 1) << (kLutBits - l);
            for (uint32_t e = lo; e < hi; ++e) a.lut[e] = (s << 8) | l;
        }
    }
    __syncthreads();
    if (tid == 0) st->dec_ok = 1;
}

// bit reader over the chunk payload (global, bounds-checked: words at or past
// `end` read as zero, so a bad stream cannot read outside it)
struct BitReader {
    const uint32_t* words;
    uint64_t pos, end;            // word index of the next refill, end (exclusive)
    unsigned long long win;       // bits MSB-aligned
    uint32_t avail;
    __device__ __forceinline__ void init(const uint32_t* w, uint64_t begin_bit, uint64_t end_word) {
        words = w;
        end = end_word;
        pos = begin_bit >> 5;
        win = 0;
        avail = 0;
        uint32_t skip = (uint32_t)(begin_bit & 31u);
        refill();
        refill();
        win <<= skip;
        avail -= skip;
    }
    __device__ __forceinline__ void refill() {
        uint32_t v = 0;
        if (pos < end) v = __ldg(words + pos);
        ++pos;
        win |= (unsigned long long)v << (32u - avail);
        avail += 32;
    }
    __device__ __forceinline__ void consume(uint32_t l) {
        win <<= l;
        avail -= l;
        if (avail < 32) refill();
    }
};

// Team-level primitives: a team is 64 threads (2 warps) with its own named
// barrier (id team + 1) decoding one chunk at a time.
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

constexpr int kTeams = 6;
constexpr int kDecBlock = kTeams * kDecThreads;        // 384
constexpr int kDecLutBits = 12;

struct DecSmem {
    uint32_t lut[1 << kDecLutBits];       // sym << 8 | len for codes of <= 12 bits, else 0
    uint32_t lim[kMaxLen + 2];            // left-justified (24-bit) end of each length's codes
    uint32_t first[kMaxLen + 2], base[kMaxLen + 2];
    uint32_t ws32[kTeams][2], ws32b[kTeams][2];
    long long ws64[kTeams][2];
    uint32_t bad[kTeams];
};

__global__ void __launch_bounds__(kDecBlock, 1) decode_kernel(DecompressArgs a) {
    __shared__ DecSmem sm;
    extern __shared__ uint4 dyn_smem[];
    const ArrayState* st = a.st;
    const int tid = threadIdx.x;
    if (!st->dec_ok) return;
    const uint8_t* in = a.in;
    const uint64_t n = st->n_out;
    if (n == 0) return;
    if (st->raw) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(in + st->off[S_PAYLOAD]);
        uint32_t* dst = reinterpret_cast<uint32_t*>(a.out);
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + tid; i < n; i += (uint64_t)gridDim.x * blockDim.x)
            dst[i] = __ldg(src + i);
        return;
    }
    const uint32_t C = rd32(in + H_C), G = rd32(in + H_G), gshift = 31 - __clz(G);
    const uint64_t nc = rd64(in + H_NCHUNKS), E = rd64(in + H_NESC), pw = rd64(in + H_PWORDS);
    const float D = __uint_as_float(rd32(in + H_D));
    const uint64_t* cword = reinterpret_cast<const uint64_t*>(in + st->off[S_CWORD]);
    const long long* anchor = reinterpret_cast<const long long*>(in + st->off[S_ANCHOR]);
    const uint64_t* cesc = reinterpret_cast<const uint64_t*>(in + st->off[S_CESC]);
    const uint16_t* sublen = reinterpret_cast<const uint16_t*>(in + st->off[S_SUBLEN]);
    const uint8_t* escs = in + st->off[S_ESC];
    const uint32_t* payload = reinterpret_cast<const uint32_t*>(in + st->off[S_PAYLOAD]);

    // block-wide: direct lookup table for codes of <= 12 bits, limits for the rest
    for (uint32_t i = tid; i < (1u << kDecLutBits); i += kDecBlock) sm.lut[i] = 0u;
    __syncthreads();
    if (tid < kMaxLen + 2) {
        const uint32_t l = tid;
        sm.first[l] = st->first[l];
        sm.base[l] = st->base[l];
        sm.lim[l] = (l >= 1 && l <= (uint32_t)kMaxLen) ? ((st->first[l] + st->count[l]) << (kMaxLen - l)) : 0u;
    }
    {
        const uint32_t m = (uint32_t)rd64(in + H_NSYM);
        for (uint32_t p = tid; p < m; p += kDecBlock) {
            // symbols in (length, symbol) order: find this position's length
            uint32_t l = 1;
            while (l < (uint32_t)kMaxLen && p >= st->base[l] + st->count[l]) ++l;
            if (l <= (uint32_t)kDecLutBits) {
                uint32_t code = st->first[l] + (p - st->base[l]);
                uint32_t lo = code << (kDecLutBits - l), hi = (code + 1) << (kDecLutBits - l);
                uint32_t v = ((uint32_t)a.by_len[p] << 8) | l;
                for (uint32_t e = lo; e < hi; ++e) sm.lut[e] = v;
            }
        }
    }
    __syncthreads();

    const int team = tid / kDecThreads, k = tid % kDecThreads;
    const int teams_active = umin32(kTeams, (uint32_t)(kTeams * 8192u) / C);
    if (team >= teams_active) return;
    uint32_t* xs = reinterpret_cast<uint32_t*>(dyn_smem) + (size_t)team * C;
    const bool vec = ((uintptr_t)a.out & 15u) == 0;
    const uint64_t stride = (uint64_t)gridDim.x * teams_active;

    for (uint64_t c = (uint64_t)blockIdx.x * teams_active + team; c < nc; c += stride) {
        const uint64_t base = c * C;
        const uint32_t cnt = (uint32_t)umin64(C, n - base);
        const uint64_t wb = cword[c], we = cword[c + 1];
        const uint64_t eb = cesc[c], ee = cesc[c + 1];
        const bool hdr_bad = (wb > we || we > pw || eb > ee || ee > E);
        const uint32_t e0 = k * G;
        const uint32_t nsym = e0 < cnt ? umin32(G, cnt - e0) : 0u;
        const uint32_t sl = sublen[c * kSubPerChunk + k];
        uint32_t tot_bits;
        const uint32_t start = team_exclusive_scan<uint32_t>(sl, sm.ws32[team], team, k, &tot_bits);
        if (hdr_bad || (uint64_t)tot_bits > 32ull * (we - wb)) {
            if (k == 0) raise_err(a.err, E_CORRUPT);
            return;
        }
        // ---- phase 1: decode the sub-stream ------------------------------------------
        BitReader br;
        br.init(payload, 32ull * wb + start, we);
        int dsum = 0;
        uint32_t nesc = 0, used = 0;
        bool bad = false;
        for (uint32_t j4 = 0; j4 < nsym; j4 += 4) {
            uint32_t sy[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (j4 + t < nsym) {
                    const uint32_t w24 = (uint32_t)(br.win >> 40);
                    uint32_t ent = sm.lut[w24 >> (kMaxLen - kDecLutBits)];
                    uint32_t sym, len;
                    if (ent) {
                        sym = ent >> 8;
                        len = ent & 255u;
                    } else {
                        len = kDecLutBits + 1;
                        while (len <= (uint32_t)kMaxLen && w24 >= sm.lim[len]) ++len;
                        if (len > (uint32_t)kMaxLen) { bad = true; len = 0; sym = 0; }
                        else sym = a.by_len[sm.base[len] + (w24 >> (kMaxLen - len)) - sm.first[len]];
                    }
                    br.consume(len);
                    used += len;
                    sy[t] = sym;
                    nesc += (sym == 0u);
                    dsum += (sym == 0u) ? 0 : (int)sym - kRadius;
                }
            }
            *reinterpret_cast<uint4*>(&xs[swz(e0 + j4, gshift)]) = make_uint4(sy[0], sy[1], sy[2], sy[3]);
        }
        bad = bad || used != sl;
        // ---- escapes and the block-wide prefix ----------------------------------------
        uint32_t tot_esc;
        const uint32_t eoff = team_exclusive_scan<uint32_t>(nesc + (bad ? 0x10000u : 0u), sm.ws32b[team], team, k,
                                                             &tot_esc);
        if ((tot_esc >> 16) || eb + tot_esc != ee) {
            if (k == 0) raise_err(a.err, E_CORRUPT);
            return;
        }
        long long sum = dsum;
        for (uint32_t t = 0; t < nesc; ++t)
            sum += *reinterpret_cast<const long long*>(escs + (uint64_t)kEscBytes * (eb + eoff + t));
        long long tot_sum;
        const long long pre = team_exclusive_scan<long long>(sum, sm.ws64[team], team, k, &tot_sum);
        // ---- phase 2: reconstruct in place -----------------------------------------
        long long q = anchor[c] + pre;
        uint64_t ecur = eb + eoff;
        for (uint32_t j4 = 0; j4 < nsym; j4 += 4) {
            uint4* slot = reinterpret_cast<uint4*>(&xs[swz(e0 + j4, gshift)]);
            uint4 s4 = *slot;
            uint32_t sy[4] = {s4.x, s4.y, s4.z, s4.w};
            uint32_t ov[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                ov[t] = 0u;
                if (j4 + t < nsym) {
                    float v;
                    if (sy[t]) {
                        q += (int)sy[t] - kRadius;
                        v = recon_f(q, D);
                    } else {
                        const uint8_t* r = escs + (uint64_t)kEscBytes * ecur++;
                        q += *reinterpret_cast<const long long*>(r);
                        v = (rd32(r + 12) & 1u) ? __uint_as_float(rd32(r + 8)) : recon_f(q, D);
                    }
                    ov[t] = __float_as_uint(v);
                }
            }
            *slot = make_uint4(ov[0], ov[1], ov[2], ov[3]);
        }
        team_sync(team);
        // ---- phase 3: coalesced store ---------------------------------------------
        float* dst = a.out + base;
        for (uint32_t e = 4 * k; e < cnt; e += 4 * kDecThreads) {
            uint4 v = *reinterpret_cast<const uint4*>(&xs[swz(e, gshift)]);
            if (vec && e + 3 < cnt) {
                *reinterpret_cast<uint4*>(dst + e) = v;
            } else {
                uint32_t vv[4] = {v.x, v.y, v.z, v.w};
                for (int j = 0; j < 4 && e + j < cnt; ++j) dst[e + j] = __uint_as_float(vv[j]);
            }
        }
        team_sync(team);
    }
}

void launch_decode_setup(const DecompressArgs* a, int k, void* stream) {
    for (int i = 0; i < k; ++i) decode_setup_kernel<<<1, kSetupThreads, 0, (cudaStream_t)stream>>>(a[i]);
}

void launch_decode(const DecompressArgs* a, int k, void* stream) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const size_t smem = (size_t)kTeams * 8192u * 4u;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    for (int i = 0; i < k; ++i) decode_kernel<<<sms, kDecBlock, smem, (cudaStream_t)stream>>>(a[i]);
}

}  // namespace szg
