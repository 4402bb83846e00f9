// sz_blocksort.cuh -- one-block stable LSD radix pass over (key, value) pairs.
// Used for the Huffman leaf order (frequency, symbol) and for the canonical
// (length, symbol) order.  Inputs are in global or shared memory (generic
// pointers); the block has NT threads.
#pragma once
#include "sz_device.cuh"

namespace szg {

struct RadixSmem {
    uint32_t cnt[256];
    uint32_t run[256];
    uint32_t tile_tot[256];
    uint32_t wc[256 * 33];     // per (digit, warp) counts, padded
    uint32_t flag;
};

// Stable pass on digit (key >> shift) & 255.  Returns false (and writes
// nothing) when every key has the same digit, so the caller keeps the input.
template <int NT>
__device__ bool radix_pass(const uint32_t* kin, const uint32_t* vin, uint32_t* kout, uint32_t* vout,
                           uint32_t m, int shift, RadixSmem& sm) {
    static_assert(NT % 32 == 0 && NT <= 1024 && NT >= 256, "block size");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 256; i += NT) sm.cnt[i] = 0;
    if (tid == 0) sm.flag = 0;
    __syncthreads();
    for (uint32_t i = tid; i < m; i += NT) atomicAdd(&sm.cnt[(kin[i] >> shift) & 255u], 1u);
    __syncthreads();
    if (tid < 32) {
        uint32_t local[8], s = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { local[j] = sm.cnt[tid * 8 + j]; s += local[j]; if (local[j] == m) sm.flag = 1; }
        uint32_t inc = warp_inclusive_scan(s);
        uint32_t run = inc - s;
#pragma unroll
        for (int j = 0; j < 8; ++j) { sm.run[tid * 8 + j] = run; run += local[j]; }
    }
    __syncthreads();
    if (sm.flag) return false;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t t0 = 0; t0 < m; t0 += NT) {
        for (int i = tid; i < 256 * 33; i += NT) sm.wc[i] = 0;
        __syncthreads();
        uint32_t i = t0 + tid;
        bool valid = i < m;
        uint32_t k = valid ? kin[i] : 0u, v = valid ? vin[i] : 0u;
        uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & lt);
        if (valid && rank == 0) sm.wc[d * 33 + warp] = __popc(peers);
        __syncthreads();
        if (tid < 256) {
            uint32_t s = 0;
            for (int w = 0; w < NT / 32; ++w) {
                uint32_t t = sm.wc[tid * 33 + w];
                sm.wc[tid * 33 + w] = s;
                s += t;
            }
            sm.tile_tot[tid] = s;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = sm.run[d] + sm.wc[d * 33 + warp] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        if (tid < 256) sm.run[tid] += sm.tile_tot[tid];
        __syncthreads();
    }
    return true;
}

// Full stable sort by key (32-bit) using up to 4 passes; result ends in
// (*kres, *vres), pointing at either buffer A or buffer B.
template <int NT>
__device__ void radix_sort(uint32_t* kA, uint32_t* vA, uint32_t* kB, uint32_t* vB, uint32_t m,
                           int key_bits, RadixSmem& sm, uint32_t** kres, uint32_t** vres) {
    uint32_t *ki = kA, *vi = vA, *ko = kB, *vo = vB;
    for (int shift = 0; shift < key_bits; shift += 8) {
        if (radix_pass<NT>(ki, vi, ko, vo, m, shift, sm)) {
            uint32_t* t = ki; ki = ko; ko = t;
            t = vi; vi = vo; vo = t;
        }
        __syncthreads();
    }
    *kres = ki;
    *vres = vi;
}

}  // namespace szg
