// k_rindex.cu -- a12-a14: the molecular-dynamics reordering of Sec. IV-B.
//
// a12  R-index keys (Fig. 3a): each coordinate is put on its own lattice
//      (the compressor's q = RNE(x / D_axis)), shifted by the per-axis
//      minimum, and the three integers are bit-interleaved with x leading
//      every 3-bit group.  At most 21 bits per axis are kept (the lowest bits
//      are dropped when the coordinates need more).  Two grid passes: the
//      per-axis lattice minimum / maximum, then the keys.
// a13  Segment-wise partial radix sort (Tables 4-5): every segment of S
//      consecutive particles is stably sorted by key >> 3p (p ignored 3-bit
//      digits), one 1024-thread block per segment, LSD passes over 8-bit
//      digits on the low 32 key bits and, only when needed, the high bits.
// a14  The permutation (position j holds original index perm[j]) is applied
//      to every field of the snapshot by a gather.  No index array is stored.
// Keys may also come from the velocities (the same kernels on fields 3..5) or
// from all six fields (Sec. IV-C, Fig. 3b): one bit of each axis per 6-bit
// digit, xx leading, at most 10 bits per axis.
#include "sz_blocksort.cuh"
#include "sz_ctx.h"

namespace szg {

constexpr int kKeyThreads = 256;
constexpr int kSortThreads = 1024;

__device__ __forceinline__ unsigned long long q_order(long long q) {
    return (unsigned long long)q ^ 0x8000000000000000ull;
}
__device__ __forceinline__ long long q_unorder(unsigned long long u) {
    return (long long)(u ^ 0x8000000000000000ull);
}

// insert two zero bits between the low 21 bits of v
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

__device__ __forceinline__ void axis_params(const ReorderArgs& a, LatticeParams P[3]) {
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const ArrayState* s = a.st[ax];
        P[ax] = make_params(range_eb_abs(a.eb[ax], a.eb_kind, s->min_key, s->max_key, s->any_finite));
    }
}

__device__ __forceinline__ long long axis_q(float x, const LatticeParams& P) {
    if (P.raw) return 0;
    long long q;
    bool v;
    lattice_q(x, P, q, v);
    return q;
}

// pass 1: per-axis minimum and maximum lattice value
__global__ void __launch_bounds__(kKeyThreads) rindex_range_kernel(ReorderArgs a) {
    LatticeParams P[3];
    axis_params(a, P);
    unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            unsigned long long u = q_order(axis_q(__ldg(a.pos[ax] + i), P[ax]));
            lo[ax] = lo[ax] < u ? lo[ax] : u;
            hi[ax] = hi[ax] > u ? hi[ax] : u;
        }
    }
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[ax], o);
            unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[ax], o);
            lo[ax] = lo[ax] < l2 ? lo[ax] : l2;
            hi[ax] = hi[ax] > h2 ? hi[ax] : h2;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&a.qrange[ax], lo[ax]);
            atomicMax(&a.qrange[3 + ax], hi[ax]);
        }
    }
}

// pass 2: keys, split into low / high 32-bit words, plus the local index
__global__ void __launch_bounds__(kKeyThreads) rindex_key_kernel(ReorderArgs a) {
    LatticeParams P[3];
    axis_params(a, P);
    long long qmin[3];
    unsigned long long umax = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        qmin[ax] = q_unorder(a.qrange[ax]);
        unsigned long long span = (unsigned long long)(q_unorder(a.qrange[3 + ax]) - qmin[ax]);
        umax = umax > span ? umax : span;
    }
    const int bits = 64 - __clzll((long long)umax);      // bit length (0 when umax == 0)
    const int drop = bits > 21 ? bits - 21 : 0;
    const int shift = 3 * (int)a.p;
    uint32_t any_hi = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long u[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
            u[ax] = (unsigned long long)(axis_q(__ldg(a.pos[ax] + i), P[ax]) - qmin[ax]) >> drop;
        unsigned long long key = (spread3(u[0]) << 2) | (spread3(u[1]) << 1) | spread3(u[2]);
        key = shift < 64 ? (key >> shift) : 0ull;
        a.key_lo[i] = (uint32_t)key;
        a.key_hi[i] = (uint32_t)(key >> 32);
        a.idx[i] = (uint32_t)(i % a.segment);
        any_hi |= (uint32_t)(key >> 32);
    }
    any_hi = __reduce_or_sync(0xffffffffu, any_hi);
    if ((threadIdx.x & 31) == 0 && any_hi) atomicOr(a.any_hi, 1u);
}

// a13: one block per segment, stable LSD radix passes (global scratch, L2-resident)
__global__ void __launch_bounds__(kSortThreads) segment_sort_kernel(ReorderArgs a) {
    __shared__ RadixSmem sm;
    const uint64_t s0 = (uint64_t)blockIdx.x * a.segment;
    const uint32_t len = (uint32_t)umin64(a.segment, a.n - s0);
    uint32_t *k0 = a.key_lo + s0, *v0 = a.idx + s0, *k1 = a.tmp_k + s0, *v1 = a.tmp_v + s0;
    for (int shift = 0; shift < 32; shift += 8) {
        if (radix_pass<kSortThreads>(k0, v0, k1, v1, len, shift, sm)) {
            uint32_t* t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
        __syncthreads();
    }
    if (*a.any_hi) {
        // sort by the high word next (stable): gather it in the current order
        uint32_t* hk = (k0 == a.key_lo + s0) ? a.tmp_k + s0 : a.key_lo + s0;
        for (uint32_t j = threadIdx.x; j < len; j += kSortThreads) hk[j] = a.key_hi[s0 + v0[j]];
        __syncthreads();
        k0 = hk;
        k1 = (hk == a.key_lo + s0) ? a.tmp_k + s0 : a.key_lo + s0;
        for (int shift = 0; shift < 32; shift += 8) {
            if (radix_pass<kSortThreads>(k0, v0, k1, v1, len, shift, sm)) {
                uint32_t* t = k0; k0 = k1; k1 = t;
                t = v0; v0 = v1; v1 = t;
            }
            __syncthreads();
        }
    }
    for (uint32_t j = threadIdx.x; j < len; j += kSortThreads) a.perm[s0 + j] = (uint32_t)(s0 + v0[j]);
}

// a14: dst[j] = src[perm[j]]
__global__ void gather_kernel(const float* __restrict__ src, float* __restrict__ dst, const uint32_t* __restrict__ perm,
                              uint64_t n) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
        dst[j] = __ldg(src + __ldg(perm + j));
}

// ---- keys from six fields (Fig. 3b) -------------------------------------------

__device__ __forceinline__ long long axis_q6(float x, const LatticeParams& P) {
    if (P.raw) return 0;
    long long q;
    bool v;
    lattice_q(x, P, q, v);
    return q;
}

__global__ void __launch_bounds__(kKeyThreads) rindex6_range_kernel(Reorder6Args a) {
    LatticeParams P[6];
#pragma unroll
    for (int ax = 0; ax < 6; ++ax) P[ax] = a.st[ax]->P;
    unsigned long long lo[6], hi[6];
#pragma unroll
    for (int ax = 0; ax < 6; ++ax) { lo[ax] = ~0ull; hi[ax] = 0ull; }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int ax = 0; ax < 6; ++ax) {
            const unsigned long long u = q_order(axis_q6(__ldg(a.pos[ax] + i), P[ax]));
            lo[ax] = lo[ax] < u ? lo[ax] : u;
            hi[ax] = hi[ax] > u ? hi[ax] : u;
        }
    }
#pragma unroll
    for (int ax = 0; ax < 6; ++ax) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo[ax], o);
            const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hi[ax], o);
            lo[ax] = lo[ax] < l2 ? lo[ax] : l2;
            hi[ax] = hi[ax] > h2 ? hi[ax] : h2;
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&a.qrange[ax], lo[ax]);
            atomicMax(&a.qrange[6 + ax], hi[ax]);
        }
    }
}

__global__ void __launch_bounds__(kKeyThreads) rindex6_key_kernel(Reorder6Args a) {
    LatticeParams P[6];
    long long qmin[6];
    unsigned long long umax = 0;
#pragma unroll
    for (int ax = 0; ax < 6; ++ax) {
        P[ax] = a.st[ax]->P;
        qmin[ax] = q_unorder(a.qrange[ax]);
        const unsigned long long span = (unsigned long long)(q_unorder(a.qrange[6 + ax]) - qmin[ax]);
        umax = umax > span ? umax : span;
    }
    const int bits = 64 - __clzll((long long)umax);
    const int drop = bits > 10 ? bits - 10 : 0, b = bits - drop;
    const int shift = 6 * (int)a.p;
    uint32_t any_hi = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long key = 0;
#pragma unroll
        for (int ax = 0; ax < 6; ++ax) {
            const unsigned long long u = (unsigned long long)(axis_q6(__ldg(a.pos[ax] + i), P[ax]) - qmin[ax]) >> drop;
            for (int k = 0; k < b; ++k) key |= ((u >> k) & 1ull) << (6 * k + (5 - ax));
        }
        key = shift < 64 ? (key >> shift) : 0ull;
        a.key_lo[i] = (uint32_t)key;
        a.key_hi[i] = (uint32_t)(key >> 32);
        a.idx[i] = (uint32_t)(i % a.segment);
        any_hi |= (uint32_t)(key >> 32);
    }
    any_hi = __reduce_or_sync(0xffffffffu, any_hi);
    if ((threadIdx.x & 31) == 0 && any_hi) atomicOr(a.any_hi, 1u);
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

void launch_rindex_keys(const ReorderArgs& a, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t grid = (uint32_t)umin64((a.n + kKeyThreads - 1) / kKeyThreads, (uint64_t)sm_count() * 8u);
    rindex_range_kernel<<<grid ? grid : 1, kKeyThreads, 0, s>>>(a);
    rindex_key_kernel<<<grid ? grid : 1, kKeyThreads, 0, s>>>(a);
}

void launch_rindex_keys6(const Reorder6Args& a, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t grid = (uint32_t)umin64((a.n + kKeyThreads - 1) / kKeyThreads, (uint64_t)sm_count() * 8u);
    rindex6_range_kernel<<<grid ? grid : 1, kKeyThreads, 0, s>>>(a);
    rindex6_key_kernel<<<grid ? grid : 1, kKeyThreads, 0, s>>>(a);
}

void launch_segment_sort(const ReorderArgs& a, void* stream) {
    const uint64_t segs = (a.n + a.segment - 1) / a.segment;
    if (segs) segment_sort_kernel<<<(uint32_t)segs, kSortThreads, 0, (cudaStream_t)stream>>>(a);
}

void launch_gather(const float* src, float* dst, const uint32_t* perm, uint64_t n, void* stream) {
    const uint32_t grid = (uint32_t)umin64((n + 255) / 256, (uint64_t)sm_count() * 8u);
    if (n) gather_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(src, dst, perm, n);
}

}  // namespace szg
