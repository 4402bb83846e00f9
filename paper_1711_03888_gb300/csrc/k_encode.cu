// k_encode.cu -- a6 + a7: Huffman encoding of the codes into chunked
// sub-streams, the chunk tables and the escape records.
//
// One 64-thread block per chunk of C elements; thread k owns sub-stream k
// (G = C/64 consecutive elements).  The chunk is staged in shared memory with
// the XOR swizzle of sz_device.cuh, so the coalesced float4 copy-in and the
// per-thread float4 walk are both conflict-free.  Pass A recomputes the
// lattice codes (a2-a3) and looks up (codeword, length); a block scan gives
// every thread its start bit, and a decoupled look-back over chunk tickets
// gives the chunk's word offset in the payload.  Pass B packs codewords
// MSB-first into a shared buffer (interior words by plain stores, the two
// boundary words of each thread by atomicOr) and the chunk is copied out
// with 128-bit stores.  Escape records are rebuilt from global memory (rare).
#include "sz_device.cuh"

namespace szg {

constexpr int kEncThreads = kSubPerChunk;     // 64
constexpr uint32_t kLookbackSpins = 1u << 22;

__device__ __forceinline__ void flush_word(uint32_t* pay, uint32_t w, uint32_t v, bool shared_word) {
    if (shared_word) atomicOr(&pay[w], v);
    else pay[w] = v;
}

__device__ void raw_copy(const CompressArgs& a) {
    const ArrayState* st = a.st;
    if (st->total_bytes > a.out_cap) return;
    uint32_t* dst = reinterpret_cast<uint32_t*>(a.out + kHeaderBytes);
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.in);
    const uint64_t n = a.n, words = (n + 3u) & ~(uint64_t)3u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = (i < n) ? __ldg(src + i) : 0u;
}

__global__ void __launch_bounds__(kEncThreads) encode_kernel(CompressArgs a) {
    extern __shared__ uint4 dyn_smem[];
    uint32_t* xs = reinterpret_cast<uint32_t*>(dyn_smem);   // C words, swizzled
    uint32_t* pay = xs + a.C;                                 // payload words of the chunk
    __shared__ uint32_t ws32[4], ws32b[4];
    __shared__ uint32_t s_c;
    __shared__ unsigned long long s_prefix;
    ArrayState* st = a.st;
    const int tid = threadIdx.x;
    if (st->raw) { raw_copy(a); return; }
    if (a.n == 0) return;
    if (tid == 0) s_c = atomicAdd(&st->ticket, 1u);
    __syncthreads();
    const uint32_t c = s_c;
    if (c >= a.n_chunks) return;

    const LatticeParams P = make_params(range_eb_abs(a.eb, a.eb_kind, st->min_key, st->max_key, st->any_finite));
    const uint32_t C = a.C, G = a.G, gshift = 31 - __clz(G);
    const uint64_t n = a.n, base = (uint64_t)c * C;
    const uint32_t cnt = (uint32_t)umin64(C, n - base);
    const float* in = a.in;
    const bool vec = ((uintptr_t)in & 15u) == 0;

    // ---- stage the chunk -------------------------------------------------------
    for (uint32_t e = 4 * tid; e < C; e += 4 * kEncThreads) {
        float4 v;
        if (vec && e + 3 < cnt) {
            v = __ldg(reinterpret_cast<const float4*>(in + base + e));
        } else {
            v.x = (e + 0 < cnt) ? __ldg(in + base + e + 0) : 0.0f;
            v.y = (e + 1 < cnt) ? __ldg(in + base + e + 1) : 0.0f;
            v.z = (e + 2 < cnt) ? __ldg(in + base + e + 2) : 0.0f;
            v.w = (e + 3 < cnt) ? __ldg(in + base + e + 3) : 0.0f;
        }
        *reinterpret_cast<float4*>(&xs[swz(e, gshift)]) = v;
    }
    __syncthreads();

    // ---- pass A: codes, lengths, escapes ------------------------------------------
    const uint32_t k = tid, e0 = k * G;
    long long qprev = 0;
    if (e0 < cnt) {
        bool vv;
        if (e0 == 0) {
            if (base > 0) lattice_q(__ldg(in + base - 1), P, qprev, vv);
        } else {
            lattice_q(__uint_as_float(xs[swz(e0 - 1, gshift)]), P, qprev, vv);
        }
    }
    __syncthreads();   // everyone has read its predecessor before slots are overwritten
    const long long anchor = qprev;
    uint32_t bits = 0, escs = 0;
    for (uint32_t m4 = 0; m4 < G; m4 += 4) {
        const uint32_t e = e0 + m4;
        uint4* slot = reinterpret_cast<uint4*>(&xs[swz(e, gshift)]);
        float4 v = *reinterpret_cast<float4*>(slot);
        float xv[4] = {v.x, v.y, v.z, v.w};
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            pk[j] = 0u;
            if (e + j < cnt) {
                long long q;
                bool vb;
                lattice_q(xv[j], P, q, vb);
                uint32_t code = make_code(q, qprev, vb);
                qprev = q;
                uint32_t ent = __ldg(&a.enc[code]);
                uint32_t len = ent & 31u;
                bits += len;
                escs += (code == 0u);
                pk[j] = ((ent >> 5) << 6) | (len << 1) | (code == 0u ? 1u : 0u);
            }
        }
        *slot = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    uint32_t chunk_bits, chunk_escs;
    const uint32_t start = block_exclusive_scan<kEncThreads>(bits, ws32, &chunk_bits);
    const uint32_t eoff = block_exclusive_scan<kEncThreads>(escs, ws32b, &chunk_escs);
    const uint32_t chunk_words = ((chunk_bits + 127u) >> 7) << 2;

    // ---- decoupled look-back: word offset of this chunk ------------------------
    if (tid == 0) {
        unsigned long long* status = a.chunk_status;
        const unsigned long long FLAG_AGG = 1ull << 62, FLAG_INC = 2ull << 62, FLAG_ERR = 3ull << 62;
        const unsigned long long VMASK = (1ull << 62) - 1;
        unsigned long long excl = 0;
        bool bad = false;
        if (c == 0) {
            st_release(&status[0], FLAG_INC | chunk_words);
        } else {
            st_release(&status[c], FLAG_AGG | chunk_words);
            int64_t j = (int64_t)c - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                unsigned long long s = ld_acquire(&status[j]);
                unsigned long long f = s & ~VMASK;
                if (f == 0ull) {
                    if (++spins > kLookbackSpins) { bad = true; break; }
                    __nanosleep(32);
                    continue;
                }
                if (f == FLAG_ERR) { bad = true; break; }
                excl += s & VMASK;
                if (f == FLAG_INC) break;
                --j;
            }
            if (bad) {
                raise_err(a.err, E_TIMEOUT);
                st_release(&status[c], FLAG_ERR);
            } else {
                st_release(&status[c], FLAG_INC | (excl + chunk_words));
            }
        }
        s_prefix = bad ? ~0ull : excl;
    }
    __syncthreads();
    const unsigned long long prefix = s_prefix;
    if (prefix == ~0ull) return;

    // ---- tables ------------------------------------------------------------------
    uint8_t* out = a.out;
    const uint64_t off_payload = st->off[S_PAYLOAD];
    const bool tables_ok = off_payload <= a.out_cap;
    const uint64_t chunk_end = off_payload + 4ull * (prefix + chunk_words);
    if (tables_ok) {
        reinterpret_cast<uint16_t*>(out + st->off[S_SUBLEN])[(uint64_t)c * kSubPerChunk + k] =
            (uint16_t)(e0 < cnt ? bits : 0u);
        if (tid == 0) {
            reinterpret_cast<uint64_t*>(out + st->off[S_CWORD])[c] = prefix;
            reinterpret_cast<long long*>(out + st->off[S_ANCHOR])[c] = anchor;
            if (c == a.n_chunks - 1) reinterpret_cast<uint64_t*>(out + st->off[S_CWORD])[c + 1] = prefix + chunk_words;
        }
    }
    if (c == a.n_chunks - 1 && tid == 0) {
        st->total_bytes = chunk_end;
        if (a.out_cap >= kHeaderBytes) {
            *reinterpret_cast<uint64_t*>(out + H_PWORDS) = prefix + chunk_words;
            *reinterpret_cast<uint64_t*>(out + H_TOTAL) = chunk_end;
        }
        if (chunk_end > a.out_cap) raise_err(a.err, E_CAPACITY);
    }
    if (!tables_ok) return;

    // ---- escape records (rare): rebuilt from global memory ---------------------
    if (escs) {
        uint8_t* esc_base = out + st->off[S_ESC] + (uint64_t)kEscBytes * (a.chunk_esc[c] + eoff);
        uint32_t idx = 0;
        for (uint32_t m1 = 0; m1 < G && e0 + m1 < cnt; ++m1) {
            if (xs[swz(e0 + m1, gshift)] & 1u) {
                uint64_t i = base + e0 + m1;
                float x = __ldg(in + i);
                long long q, qp = 0;
                bool vb, vv;
                lattice_q(x, P, q, vb);
                if (i > 0) lattice_q(__ldg(in + i - 1), P, qp, vv);
                uint8_t* r = esc_base + (uint64_t)kEscBytes * idx++;
                *reinterpret_cast<long long*>(r) = q - qp;
                *reinterpret_cast<uint32_t*>(r + 8) = vb ? __float_as_uint(x) : 0u;
                *reinterpret_cast<uint32_t*>(r + 12) = vb ? 1u : 0u;
            }
        }
    }

    // ---- pass B: pack --------------------------------------------------------------
    for (uint32_t w = tid; w < chunk_words; w += kEncThreads) pay[w] = 0u;
    __syncthreads();
    {
        uint32_t word = start >> 5, fill = start & 31u, cur = 0u;
        bool first = true;
        for (uint32_t m4 = 0; m4 < G; m4 += 4) {
            uint4 p4 = *reinterpret_cast<const uint4*>(&xs[swz(e0 + m4, gshift)]);
            uint32_t pk[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t len = (pk[j] >> 1) & 31u;
                if (len == 0u) continue;
                uint32_t cw = pk[j] >> 6;
                uint32_t room = 32u - fill;
                if (len < room) {
                    cur |= cw << (room - len);
                    fill += len;
                } else {
                    uint32_t spill = len - room;          // 0..23
                    cur |= cw >> spill;
                    flush_word(pay, word, cur, first);
                    first = false;
                    ++word;
                    cur = spill ? (cw << (32u - spill)) : 0u;
                    fill = spill;
                }
            }
        }
        if (fill) flush_word(pay, word, cur, true);
    }
    __syncthreads();
    if (chunk_end <= a.out_cap) {
        uint4* dst = reinterpret_cast<uint4*>(out + off_payload + 4ull * prefix);
        const uint4* src = reinterpret_cast<const uint4*>(pay);
        for (uint32_t w4 = tid; w4 < chunk_words / 4; w4 += kEncThreads) dst[w4] = src[w4];
    }
}

void launch_encode(const CompressArgs* a, int k, void* stream) {
    for (int i = 0; i < k; ++i) {
        if (a[i].n == 0) continue;
        size_t smem = (size_t)a[i].C * 4u + ((size_t)a[i].C * 3u / 4u + 4u) * 4u;
        static size_t configured = 0;
        if (smem > configured) {
            cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            configured = smem;
        }
        encode_kernel<<<a[i].n_chunks, kEncThreads, smem, (cudaStream_t)stream>>>(a[i]);
    }
}

}  // namespace szg
