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

// bit reader over the chunk payload (global, bounds-checked)
struct BitReader {
    const uint32_t* words;
    uint64_t pos, end;            // word index of the next refill, end (exclusive)
    unsigned long long win;       // bits MSB-aligned
    uint32_t avail;
    bool bad;
    __device__ __forceinline__ void init(const uint32_t* w, uint64_t begin_bit, uint64_t end_word) {
        words = w;
        end = end_word;
        pos = begin_bit >> 5;
        win = 0;
        avail = 0;
        bad = false;
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

__global__ void __launch_bounds__(kDecThreads) decode_kernel(DecompressArgs a) {
    extern __shared__ uint4 dyn_smem[];
    uint32_t* xs = reinterpret_cast<uint32_t*>(dyn_smem);
    __shared__ uint32_t ws32[4], ws32b[4];
    __shared__ unsigned long long ws64[4];
    __shared__ uint32_t s_first[kMaxLen + 2], s_count[kMaxLen + 2], s_base[kMaxLen + 2];
    __shared__ uint32_t s_bad, s_bad_hdr;
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
    for (int l = tid; l < kMaxLen + 2; l += kDecThreads) {
        s_first[l] = st->first[l];
        s_count[l] = st->count[l];
        s_base[l] = st->base[l];
    }
    const bool vec = ((uintptr_t)a.out & 15u) == 0;
    __syncthreads();

    for (uint64_t c = blockIdx.x; c < nc; c += gridDim.x) {
        const uint64_t base = c * C;
        const uint32_t cnt = (uint32_t)umin64(C, n - base);
        const uint64_t wb = cword[c], we = cword[c + 1];
        const uint64_t eb = cesc[c], ee = cesc[c + 1];
        if (tid == 0) {
            s_bad_hdr = (wb > we || we > pw || eb > ee || ee > E) ? 1u : 0u;
            s_bad = 0u;
        }
        const uint32_t k = tid, e0 = k * G;
        const uint32_t nsym = e0 < cnt ? min(G, cnt - e0) : 0u;
        const uint32_t sl = sublen[c * kSubPerChunk + k];
        uint32_t tot_bits;
        const uint32_t start = block_exclusive_scan<kDecThreads>(sl, ws32, &tot_bits);
        if (s_bad_hdr || (uint64_t)tot_bits > 32ull * (we - wb)) {
            if (tid == 0) raise_err(a.err, E_CORRUPT);
            return;
        }
        // ---- phase 1: decode the sub-stream, 4 symbols per shared store --------------
        BitReader br;
        br.init(payload, 32ull * wb + start, we);
        int dsum = 0;
        uint32_t nesc = 0, used = 0;
        bool bad = false;
        for (uint32_t j4 = 0; j4 < nsym; j4 += 4) {
            uint32_t sy[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (j4 + t < nsym && !bad) {
                    uint32_t top = (uint32_t)(br.win >> (64 - kLutBits));
                    uint32_t ent = __ldg(a.lut + top);
                    uint32_t sym, len;
                    if (ent) {
                        sym = ent >> 8;
                        len = ent & 255u;
                    } else {
                        sym = 0; len = 0;
                        for (uint32_t l = kLutBits + 1; l <= (uint32_t)kMaxLen; ++l) {
                            uint32_t code = (uint32_t)(br.win >> (64 - l));
                            uint32_t d = code - s_first[l];
                            if (d < s_count[l]) { sym = a.by_len[s_base[l] + d]; len = l; break; }
                        }
                        if (!len) bad = true;
                    }
                    br.consume(len);
                    used += len;
                    sy[t] = sym;
                    if (sym == 0u) ++nesc;
                    else dsum += (int)sym - kRadius;
                }
            }
            *reinterpret_cast<uint4*>(&xs[swz(e0 + j4, gshift)]) = make_uint4(sy[0], sy[1], sy[2], sy[3]);
        }
        bad = bad || used != sl;
        // ---- escapes and the block-wide prefix ----------------------------------------
        if (bad) atomicOr(&s_bad, 1u);
        uint32_t tot_esc;
        const uint32_t eoff = block_exclusive_scan<kDecThreads>(nesc, ws32b, &tot_esc);
        if (s_bad || eb + tot_esc != ee) {
            if (tid == 0) raise_err(a.err, E_CORRUPT);
            return;
        }
        long long sum = dsum;
        for (uint32_t t = 0; t < nesc; ++t)
            sum += *reinterpret_cast<const long long*>(escs + (uint64_t)kEscBytes * (eb + eoff + t));
        long long tot_sum;
        const long long pre = block_exclusive_scan<kDecThreads, long long>(sum, reinterpret_cast<long long*>(ws64), &tot_sum);
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
        __syncthreads();
        // ---- phase 3: coalesced store ---------------------------------------------
        float* dst = a.out + base;
        for (uint32_t e = 4 * tid; e < cnt; e += 4 * kDecThreads) {
            uint4 v = *reinterpret_cast<const uint4*>(&xs[swz(e, gshift)]);
            if (vec && e + 3 < cnt) {
                *reinterpret_cast<uint4*>(dst + e) = v;
            } else {
                uint32_t vv[4] = {v.x, v.y, v.z, v.w};
                for (int j = 0; j < 4 && e + j < cnt; ++j) dst[e + j] = __uint_as_float(vv[j]);
            }
        }
        __syncthreads();
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
    const size_t smem = 16384u * 4u;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    for (int i = 0; i < k; ++i) decode_kernel<<<sms * 8, kDecThreads, smem, (cudaStream_t)stream>>>(a[i]);
}

}  // namespace szg
