// sz_quant.cuh -- a2-a4 body: one chunk of value -> lattice, last-value
// prediction on the lattice, linear-scaling quantization into 2^16 codes
// (Sec. IV-A) and the code histogram, for a block of 256 threads.
//
// Each of the 8 warps owns a contiguous span of C/8 elements and walks it
// 256 elements per step (two 128-element groups, both float4 loads issued
// first), carrying the last lattice value from lane 31 to lane 0 of the next
// group, so only the first group of a span recomputes a predecessor.  The
// common case runs in 32-bit arithmetic: a refined FP32 candidate (x*inv
// corrected by one fma residual) is exact except within 2^-20 of a
// half-integer, which the residual test detects; any warp step holding such
// an element, or a candidate beyond 2^22, takes the general binary64 path
// for that step.  Codes near the centre go to a shared-memory window of the
// histogram, the rest to global atomics.  When `codes` is set the u16 codes
// are stored for the encoder.  The chunk's escape count is recorded and the
// encoder's look-back word re-armed.  quant_chunk reads the input from global
// memory; quant_chunk_staged from a shared-memory stage that the persistent
// loop (quant_array_staged) fills for the next chunk while this one runs.
// With LCF = true the prediction is the original SZ's linear curve fitting
// (Sec. IV-A): the code carries the second difference q_i - 2 q_{i-1} +
// q_{i-2}, so each warp also carries q_{i-2} from group to group.
#pragma once
#include "sz_device.cuh"

namespace szg {

constexpr int kQuantThreads = 256;
// Shared histogram window: codes kWinLo .. kWinLo + kWin - 1 (deltas within
// +-8192), two 16-bit counters per word (kWinWords words, 32 KB).  A block
// flushes it into the global histogram before a counter can wrap: after at
// most 65535 elements (quant_flush_every chunks).  Measured on GB300 (2^27
// elements, quantize ms, positions / velocities): 32-bit counters over 8192
// codes 0.50 / 0.29; 16-bit counters over 16384 codes 0.33 / 0.32 -- position
// data puts ~3 % of its codes beyond +-4096, and every one of those costs a
// divergent global atomic.
constexpr int kWin = 16384;
constexpr int kWinWords = kWin / 2;
constexpr uint32_t kWinLo = kRadius - kWin / 2;
__host__ __device__ constexpr uint32_t quant_flush_every(uint32_t C) { return 65535u / C; }

// dynamic shared memory of the staged quantize loop: NSTAGE stages of C + 4 floats.
// Measured on GB300 (2^27 elements, C = 4096): the stand-alone kernel (64
// registers) runs 4 blocks per SM with one stage (48 KB per block) against 3
// with two, 0.306 vs 0.329 ms; the batched kernel does the same under a
// launch bound for four blocks.
constexpr size_t quant_stage_bytes(uint32_t C, int NSTAGE = 2) { return (size_t)NSTAGE * 4u * ((size_t)C + 4u); }

// The escape code (0) is not added here: every escape would hit the same
// global counter, and at rel eb 1e-5 a position field escapes ~3 % of its
// elements.  The chunk's escape count goes to gh[0] once per chunk instead.
__device__ __forceinline__ void hist_add(uint32_t code, uint32_t* sh, uint32_t* gh) {
    const uint32_t w = code - kWinLo;
    if (w < (uint32_t)kWin) atomicAdd(&sh[w >> 1], 1u << ((w & 1u) << 4));
    else if (code != 0u) atomicAdd(&gh[code], 1u);
}

// FP32 fast path: returns false when the element needs the general path.
__device__ __forceinline__ bool lattice_fast32(float x, const LatticeParams& P, int& q, bool& verb) {
    float t1 = x * P.inv;
    float e = fmaf(-t1, P.D, x);
    float t = fmaf(e, P.inv, t1);
    // nearest integer, ties to even, by one rounded add of 1.5 * 2^23: for
    // |t| < 2^22 (the only case this path accepts) the sum's low mantissa
    // bits hold the integer, and subtracting the constant again is exact
    const float big = __fadd_rn(t, 12582912.0f);
    const float qc = __fsub_rn(big, 12582912.0f);
    q = __float_as_int(big) - 0x4B400000;
    float r = fmaf(-qc, P.D, x);
    float xr = __fmul_rn(qc, P.D);
    verb = fabsf(__fsub_rn(x, xr)) > P.ebf;
    return (fabsf(r) <= P.thr_lo) & (fabsf(t) < 4194304.0f);
}

__device__ __forceinline__ uint32_t code32(int q, int qprev, bool verb) {
    int d = q - qprev;
    return (verb || (uint32_t)(d + (kRadius - 1)) > (uint32_t)(2 * kRadius - 2)) ? 0u : (uint32_t)(d + kRadius);
}

__device__ __forceinline__ void hist_window_zero(uint32_t* sh) {
    for (int i = threadIdx.x; i < kWinWords; i += kQuantThreads) sh[i] = 0u;
}

// adds the window into the global histogram and clears it (callers
// synchronize the block before and after)
__device__ __forceinline__ void hist_window_flush(uint32_t* sh, uint32_t* gh) {
    for (int i = threadIdx.x; i < kWinWords; i += kQuantThreads) {
        const uint32_t v = sh[i];
        if (v & 0xffffu) atomicAdd(&gh[kWinLo + 2 * i], v & 0xffffu);
        if (v >> 16) atomicAdd(&gh[kWinLo + 2 * i + 1], v >> 16);
        sh[i] = 0u;
    }
}

template <bool STORE, bool LCF = false>
__device__ void quant_chunk(const CompressArgs& a, const LatticeParams& P, uint32_t c, uint32_t* sh,
                            uint32_t* s_esc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* in = a.in;
    const bool vec = ((uintptr_t)in & 15u) == 0;
    const bool fast_ok = P.fast != 0;
    const uint64_t n = a.n;
    const uint32_t span = a.C / 8;
    uint16_t* codes = a.codes;
    const uint64_t s0 = (uint64_t)c * a.C + (uint64_t)warp * span;
    const uint64_t s1 = umin64(n, s0 + span);
    uint32_t esc = 0;
    long long carry = 0, carry2 = 0;     // q_{s0-1}, and q_{s0-2} for LCF
    if (s0 < s1 && s0 > 0 && lane == 0) {
        bool vv;
        lattice_q(__ldg(in + s0 - 1), P, carry, vv);
        if (LCF && s0 > 1) lattice_q(__ldg(in + s0 - 2), P, carry2, vv);
    }
    carry = __shfl_sync(0xffffffffu, carry, 0);
    if (LCF) carry2 = __shfl_sync(0xffffffffu, carry2, 0);
    for (uint64_t ib = s0; ib < s1; ib += 256) {
        float xg[2][4];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const uint64_t i = ib + 128 * g + 4 * (uint64_t)lane;
            if (vec && ib + 128 * g + 128 <= s1) {
                float4 v = __ldg(reinterpret_cast<const float4*>(in + i));
                xg[g][0] = v.x; xg[g][1] = v.y; xg[g][2] = v.z; xg[g][3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) xg[g][j] = (i + j < s1) ? __ldg(in + i + j) : 0.0f;
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const uint64_t i0 = ib + 128 * g;
            if (i0 >= s1) break;
            const uint64_t i = i0 + 4 * (uint64_t)lane;
            const bool full = (i0 + 128 <= s1);
            float x[4] = {xg[g][0], xg[g][1], xg[g][2], xg[g][3]};
            uint32_t cd[4];
            int q32[4];
            bool vb[4];
            bool ok = fast_ok;
#pragma unroll
            for (int j = 0; j < 4; ++j) ok &= lattice_fast32(x[j], P, q32[j], vb[j]);
            if (LCF) {
                // second differences: delta = (q - q1) - (q1 - q2), so the LV code
                // builders apply to the first differences
                if (__all_sync(0xffffffffu, ok) && carry >= -(1ll << 28) && carry <= (1ll << 28) &&
                    carry2 >= -(1ll << 28) && carry2 <= (1ll << 28)) {
                    int qp = __shfl_up_sync(0xffffffffu, q32[3], 1);
                    int qpp = __shfl_up_sync(0xffffffffu, q32[2], 1);
                    if (lane == 0) { qp = (int)carry; qpp = (int)carry2; }
                    cd[0] = code32(q32[0] - qp, qp - qpp, vb[0]);
                    cd[1] = code32(q32[1] - q32[0], q32[0] - qp, vb[1]);
                    cd[2] = code32(q32[2] - q32[1], q32[1] - q32[0], vb[2]);
                    cd[3] = code32(q32[3] - q32[2], q32[2] - q32[1], vb[3]);
                    carry = __shfl_sync(0xffffffffu, q32[3], 31);
                    carry2 = __shfl_sync(0xffffffffu, q32[2], 31);
                } else {
                    long long q[4];
                    bool v2[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], v2[j]);
                    long long qp = __shfl_up_sync(0xffffffffu, q[3], 1);
                    long long qpp = __shfl_up_sync(0xffffffffu, q[2], 1);
                    if (lane == 0) { qp = carry; qpp = carry2; }
                    cd[0] = make_code(q[0] - qp, qp - qpp, v2[0]);
                    cd[1] = make_code(q[1] - q[0], q[0] - qp, v2[1]);
                    cd[2] = make_code(q[2] - q[1], q[1] - q[0], v2[2]);
                    cd[3] = make_code(q[3] - q[2], q[2] - q[1], v2[3]);
                    carry = __shfl_sync(0xffffffffu, q[3], 31);
                    carry2 = __shfl_sync(0xffffffffu, q[2], 31);
                }
            } else if (__all_sync(0xffffffffu, ok) && carry >= -(1ll << 30) && carry <= (1ll << 30)) {
                int qp = __shfl_up_sync(0xffffffffu, q32[3], 1);
                if (lane == 0) qp = (int)carry;
                cd[0] = code32(q32[0], qp, vb[0]);
                cd[1] = code32(q32[1], q32[0], vb[1]);
                cd[2] = code32(q32[2], q32[1], vb[2]);
                cd[3] = code32(q32[3], q32[2], vb[3]);
                carry = __shfl_sync(0xffffffffu, q32[3], 31);
            } else {
                long long q[4];
                bool v2[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], v2[j]);
                long long qp = __shfl_up_sync(0xffffffffu, q[3], 1);
                if (lane == 0) qp = carry;
                cd[0] = make_code(q[0], qp, v2[0]);
                cd[1] = make_code(q[1], q[0], v2[1]);
                cd[2] = make_code(q[2], q[1], v2[2]);
                cd[3] = make_code(q[3], q[2], v2[3]);
                // only full groups continue, so lane 31's q[3] is the last element
                carry = __shfl_sync(0xffffffffu, q[3], 31);
            }
            if (full) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    esc += (cd[j] == 0u);
                    hist_add(cd[j], sh, a.hist);
                }
                if (STORE) {
                    uint2 pk = make_uint2(cd[0] | (cd[1] << 16), cd[2] | (cd[3] << 16));
                    *reinterpret_cast<uint2*>(codes + i) = pk;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i + j < s1) {
                        esc += (cd[j] == 0u);
                        hist_add(cd[j], sh, a.hist);
                        if (STORE) codes[i + j] = (uint16_t)cd[j];
                    }
            }
        }
    }
    esc = warp_reduce_sum(esc);
    if (lane == 0) s_esc[warp] = esc;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kQuantThreads / 32; ++w) t += s_esc[w];
        a.chunk_esc[c] = t;
        if (t) atomicAdd(&a.hist[0], t);     // the escapes hist_add leaves out
        a.chunk_status[c] = 0ull;
    }
    __syncthreads();
}

template <bool STORE, bool LCF = false>
__device__ void quant_chunk_staged(const CompressArgs& a, const LatticeParams& P, uint32_t c, const float* stage,
                                   uint32_t* sh, uint32_t* s_esc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t cbase = (uint64_t)c * a.C;
    const float* sx = stage + 4;           // sx[o] = x[cbase + o]; sx[-4 .. -1] = the elements before the chunk
    const bool fast_ok = P.fast != 0;
    const uint32_t span = a.C / 8;
    uint16_t* codes = a.codes + cbase;
    // chunk-relative offsets: this warp's span is s0 .. s1 - 1
    const uint32_t s0 = (uint32_t)warp * span;
    const uint32_t s1 = (uint32_t)umin64(a.n - cbase, (uint64_t)s0 + span);
    uint32_t esc = 0;
    long long carry = 0, carry2 = 0;     // q_{s0-1}, and q_{s0-2} for LCF
    if (s0 < s1 && cbase + s0 > 0 && lane == 0) {
        bool vv;
        lattice_q(sx[(int)s0 - 1], P, carry, vv);
        if (LCF && cbase + s0 > 1) lattice_q(sx[(int)s0 - 2], P, carry2, vv);   // the stage holds 4 before the chunk
    }
    carry = __shfl_sync(0xffffffffu, carry, 0);
    if (LCF) carry2 = __shfl_sync(0xffffffffu, carry2, 0);
    for (uint32_t ib = s0; ib < s1; ib += 256) {
        float xg[2][4];
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const uint32_t i = ib + 128 * g + 4 * lane;
            if (ib + 128 * g + 128 <= s1) {
                float4 v = *reinterpret_cast<const float4*>(sx + i);
                xg[g][0] = v.x; xg[g][1] = v.y; xg[g][2] = v.z; xg[g][3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) xg[g][j] = (i + j < s1) ? sx[i + j] : 0.0f;
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const uint32_t i0 = ib + 128 * g;
            if (i0 >= s1) break;
            const uint32_t i = i0 + 4 * lane;
            const bool full = (i0 + 128 <= s1);
            float x[4] = {xg[g][0], xg[g][1], xg[g][2], xg[g][3]};
            uint32_t cd[4];
            int q32[4];
            bool vb[4];
            bool ok = fast_ok;
#pragma unroll
            for (int j = 0; j < 4; ++j) ok &= lattice_fast32(x[j], P, q32[j], vb[j]);
            if (LCF) {
                // second differences: delta = (q - q1) - (q1 - q2), so the LV code
                // builders apply to the first differences
                if (__all_sync(0xffffffffu, ok) && carry >= -(1ll << 28) && carry <= (1ll << 28) &&
                    carry2 >= -(1ll << 28) && carry2 <= (1ll << 28)) {
                    int qp = __shfl_up_sync(0xffffffffu, q32[3], 1);
                    int qpp = __shfl_up_sync(0xffffffffu, q32[2], 1);
                    if (lane == 0) { qp = (int)carry; qpp = (int)carry2; }
                    cd[0] = code32(q32[0] - qp, qp - qpp, vb[0]);
                    cd[1] = code32(q32[1] - q32[0], q32[0] - qp, vb[1]);
                    cd[2] = code32(q32[2] - q32[1], q32[1] - q32[0], vb[2]);
                    cd[3] = code32(q32[3] - q32[2], q32[2] - q32[1], vb[3]);
                    carry = __shfl_sync(0xffffffffu, q32[3], 31);
                    carry2 = __shfl_sync(0xffffffffu, q32[2], 31);
                } else {
                    long long q[4];
                    bool v2[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], v2[j]);
                    long long qp = __shfl_up_sync(0xffffffffu, q[3], 1);
                    long long qpp = __shfl_up_sync(0xffffffffu, q[2], 1);
                    if (lane == 0) { qp = carry; qpp = carry2; }
                    cd[0] = make_code(q[0] - qp, qp - qpp, v2[0]);
                    cd[1] = make_code(q[1] - q[0], q[0] - qp, v2[1]);
                    cd[2] = make_code(q[2] - q[1], q[1] - q[0], v2[2]);
                    cd[3] = make_code(q[3] - q[2], q[2] - q[1], v2[3]);
                    carry = __shfl_sync(0xffffffffu, q[3], 31);
                    carry2 = __shfl_sync(0xffffffffu, q[2], 31);
                }
            } else if (__all_sync(0xffffffffu, ok) && carry >= -(1ll << 30) && carry <= (1ll << 30)) {
                int qp = __shfl_up_sync(0xffffffffu, q32[3], 1);
                if (lane == 0) qp = (int)carry;
                cd[0] = code32(q32[0], qp, vb[0]);
                cd[1] = code32(q32[1], q32[0], vb[1]);
                cd[2] = code32(q32[2], q32[1], vb[2]);
                cd[3] = code32(q32[3], q32[2], vb[3]);
                carry = __shfl_sync(0xffffffffu, q32[3], 31);
            } else {
                long long q[4];
                bool v2[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], v2[j]);
                long long qp = __shfl_up_sync(0xffffffffu, q[3], 1);
                if (lane == 0) qp = carry;
                cd[0] = make_code(q[0], qp, v2[0]);
                cd[1] = make_code(q[1], q[0], v2[1]);
                cd[2] = make_code(q[2], q[1], v2[2]);
                cd[3] = make_code(q[3], q[2], v2[3]);
                // only full groups continue, so lane 31's q[3] is the last element
                carry = __shfl_sync(0xffffffffu, q[3], 31);
            }
            if (full) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    esc += (cd[j] == 0u);
                    hist_add(cd[j], sh, a.hist);
                }
                if (STORE) {
                    uint2 pk = make_uint2(cd[0] | (cd[1] << 16), cd[2] | (cd[3] << 16));
                    *reinterpret_cast<uint2*>(codes + i) = pk;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i + j < s1) {
                        esc += (cd[j] == 0u);
                        hist_add(cd[j], sh, a.hist);
                        if (STORE) codes[i + j] = (uint16_t)cd[j];
                    }
            }
        }
    }
    esc = warp_reduce_sum(esc);
    if (lane == 0) s_esc[warp] = esc;
    __syncthreads();
    if (tid == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kQuantThreads / 32; ++w) t += s_esc[w];
        a.chunk_esc[c] = t;
        if (t) atomicAdd(&a.hist[0], t);     // the escapes hist_add leaves out
        a.chunk_status[c] = 0ull;
    }
    __syncthreads();
}


// Staged input: the chunk's elements and the four before it, in shared memory
// (C + 4 floats).  quant_issue starts the asynchronous copies of chunk cc into
// `stage` (16-byte cp.async pieces, the last < 4 elements by plain loads) and
// commits them as one group; the caller waits and synchronizes the block
// before quant_chunk_staged reads the stage.  Needs a 16-byte aligned input.
__device__ __forceinline__ void quant_issue(const CompressArgs& a, uint32_t cc, float* stage) {
    const uint64_t cb = (uint64_t)cc * a.C;
    const uint64_t e0 = cc ? cb - 4 : 0, e1 = umin64(a.n, cb + a.C);
    float* sx = stage + 4;
    const uint32_t nvec = (uint32_t)((e1 - e0) / 4);
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(sx + (e0 - cb));   // e0 - cb is 0 or -4
    for (uint32_t i = threadIdx.x; i < nvec; i += kQuantThreads)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s_base + 16u * i),
                     "l"(__cvta_generic_to_global(a.in + e0 + 4 * (uint64_t)i))
                     : "memory");
    for (uint64_t e = e0 + 4 * (uint64_t)nvec + threadIdx.x; e < e1; e += kQuantThreads) sx[e - cb] = __ldg(a.in + e);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The same loop reading the input from global memory (unaligned input).
template <bool STORE, bool LCF = false>
__device__ __forceinline__ void quant_array_global(const CompressArgs& a, const LatticeParams& P, uint32_t first,
                                                   uint32_t step, uint32_t* sh, uint32_t* s_esc) {
    uint32_t since = 0;
    for (uint32_t c = first; c < a.n_chunks; c += step) {
        quant_chunk<STORE, LCF>(a, P, c, sh, s_esc);
        if (++since == quant_flush_every(a.C)) {
            hist_window_flush(sh, a.hist);
            __syncthreads();
            since = 0;
        }
    }
}

// The persistent quantize loop of one array over chunks first, first + step,
// ...: with two stages chunk c + step is copied into one while chunk c is
// quantized from the other; with one stage the copy of each chunk waits for
// the previous chunk (other resident blocks cover the latency).  stage:
// NSTAGE (C + 4) floats, 16-byte aligned.
template <bool STORE, bool LCF = false, int NSTAGE = 2>
__device__ __forceinline__ void quant_array_staged(const CompressArgs& a, const LatticeParams& P, uint32_t first,
                                                   uint32_t step, float* stage, uint32_t* sh, uint32_t* s_esc) {
    static_assert(NSTAGE == 1 || NSTAGE == 2, "stages");
    if (NSTAGE == 1) {
        uint32_t since = 0;
        for (uint32_t c = first; c < a.n_chunks; c += step) {
            quant_issue(a, c, stage);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            __syncthreads();          // chunk c is staged
            quant_chunk_staged<STORE, LCF>(a, P, c, stage, sh, s_esc);   // ends with a block barrier
            if (++since == quant_flush_every(a.C)) {
                hist_window_flush(sh, a.hist);
                __syncthreads();
                since = 0;
            }
        }
        return;
    }
    float* buf[2] = {stage, stage + a.C + 4};
    uint32_t c = first, since = 0;
    if (c < a.n_chunks) quant_issue(a, c, buf[0]);
    for (int b = 0; c < a.n_chunks; b ^= 1) {
        const uint32_t cn = c + step;
        if (cn < a.n_chunks) quant_issue(a, cn, buf[b ^ 1]);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();          // chunk c is staged (every thread's pieces)
        quant_chunk_staged<STORE, LCF>(a, P, c, buf[b], sh, s_esc);   // ends with a block barrier
        if (++since == quant_flush_every(a.C)) {
            hist_window_flush(sh, a.hist);
            __syncthreads();
            since = 0;
        }
        c = cn;
    }
}

}  // namespace szg
