// sz_range.cuh -- a1 body: value range of the finite elements of one array
// (Sec. III, "value-range-based relative error bound": eb_abs = eb_rel *
// (max - min)).  Block `bid` of `nblocks` takes a grid-stride share with four
// float4 loads in flight per thread; per-block min/max keys go to device
// atomics and the array's last block publishes the result and re-arms the
// accumulators.  The same blocks zero the array's code histogram.
#pragma once
#include "sz_device.cuh"

namespace szg {

template <int NT>
__device__ __forceinline__ void range_body(const CompressArgs& a, uint32_t bid, uint32_t nblocks) {
    __shared__ uint32_t s_min[NT / 32], s_max[NT / 32], s_any[NT / 32];
    __shared__ bool s_last;
    ArrayState* st = a.st;
    const uint32_t tid = threadIdx.x;
    const uint64_t gtid = (uint64_t)bid * NT + tid;
    const uint64_t gstride = (uint64_t)nblocks * NT;
    for (uint64_t i = gtid; i < (uint64_t)kNumCodes; i += gstride) a.hist[i] = 0u;

    uint32_t kmin = 0xffffffffu, kmax = 0u, any = 0u;
    if (a.eb_kind == 1 && a.n > 0) {
        const float* in = a.in;
        uint64_t n = a.n;
        uint64_t head = 0;
        if (((uintptr_t)in & 15u) == 0) {
            const float4* v4 = reinterpret_cast<const float4*>(in);
            const uint64_t n4 = n >> 2;
            // four 16-byte loads in flight per thread
            for (uint64_t i = gtid; i < n4; i += 4 * gstride) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = (i + u * gstride < n4) ? __ldg(v4 + i + u * gstride) : __ldg(v4 + i);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float e[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (finite_f(e[j])) {
                            uint32_t k = float_key(e[j]);
                            kmin = min(kmin, k);
                            kmax = max(kmax, k);
                            any = 1u;
                        }
                }
            }
            head = n4 << 2;
        }
        for (uint64_t i = head + gtid; i < n; i += gstride) {
            float x = __ldg(in + i);
            if (finite_f(x)) {
                uint32_t k = float_key(x);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
                any = 1u;
            }
        }
    }
    // block reduce
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        any |= __shfl_xor_sync(0xffffffffu, any, o);
    }
    if ((tid & 31) == 0) { s_min[tid >> 5] = kmin; s_max[tid >> 5] = kmax; s_any[tid >> 5] = any; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NT / 32; ++w) {
            kmin = min(kmin, s_min[w]);
            kmax = max(kmax, s_max[w]);
            any |= s_any[w];
        }
        if (any) {
            atomicMin(&st->acc_min, kmin);
            atomicMax(&st->acc_max, kmax);
            atomicOr(&st->acc_any, 1u);
        }
        __threadfence();
        s_last = (atomicAdd(&st->acc_blocks, 1u) == nblocks - 1);
    }
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        const uint32_t kmin2 = atomicExch(&st->acc_min, 0xffffffffu);
        const uint32_t kmax2 = atomicExch(&st->acc_max, 0u);
        const uint32_t any2 = atomicExch(&st->acc_any, 0u);
        st->min_key = kmin2;
        st->max_key = kmax2;
        st->any_finite = any2;
        st->P = make_params(range_eb_abs(a.eb, a.eb_kind, kmin2, kmax2, any2));
        st->acc_blocks = 0u;
        st->cb_done = 0u;
        st->range_done = 1u;
    }
}

}  // namespace szg
