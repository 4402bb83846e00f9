// k_quant.cu -- a2-a4: value -> lattice, last-value prediction on the
// lattice, linear-scaling quantization into 2^16 codes (Sec. IV-A) and the
// code histogram.  Persistent blocks walk chunks; each thread takes one
// float4 per 1024-element step; the predecessor's lattice value comes from
// the neighbouring lane (lane 0 recomputes it from memory).  Codes near the
// centre land in a shared-memory window of the histogram, the rest go to
// global atomics.  Per chunk the kernel records its escape count and re-arms
// the encoder's look-back word.
#include "sz_device.cuh"

namespace szg {

constexpr int kQuantThreads = 256;
constexpr int kWin = 4096;                 // shared histogram window (codes 30720..34815)
constexpr uint32_t kWinLo = kRadius - kWin / 2;

__device__ __forceinline__ void hist_add(uint32_t code, uint32_t* sh, uint32_t* gh) {
    uint32_t w = code - kWinLo;
    if (w < (uint32_t)kWin) atomicAdd(&sh[w], 1u);
    else atomicAdd(&gh[code], 1u);
}

__global__ void __launch_bounds__(kQuantThreads) quant_kernel(CompressArgs a) {
    __shared__ uint32_t sh[kWin];
    __shared__ uint32_t s_esc[kQuantThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ArrayState* st = a.st;
    LatticeParams P = make_params(range_eb_abs(a.eb, a.eb_kind, st->min_key, st->max_key, st->any_finite));
    if (P.raw || a.n == 0) return;
    for (int i = tid; i < kWin; i += kQuantThreads) sh[i] = 0u;
    __syncthreads();

    const float* in = a.in;
    const bool vec = ((uintptr_t)in & 15u) == 0;
    const uint64_t n = a.n;
    for (uint32_t c = blockIdx.x; c < a.n_chunks; c += gridDim.x) {
        const uint64_t base = (uint64_t)c * a.C;
        const uint64_t end = min(n, base + a.C);
        uint32_t esc = 0;
        for (uint64_t i0 = base; i0 < end; i0 += 4 * kQuantThreads) {
            const uint64_t i = i0 + 4 * (uint64_t)tid;
            float x[4];
            if (vec && i + 3 < end) {
                float4 v = __ldg(reinterpret_cast<const float4*>(in + i));
                x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) x[j] = (i + j < end) ? __ldg(in + i + j) : 0.0f;
            }
            long long q[4];
            bool vb[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) lattice_q(x[j], P, q[j], vb[j]);
            long long qprev = __shfl_up_sync(0xffffffffu, q[3], 1);
            if (lane == 0) {
                qprev = 0;
                if (i > 0 && i < end) {
                    bool vv;
                    lattice_q(__ldg(in + i - 1), P, qprev, vv);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (i + j < end) {
                    uint32_t code = make_code(q[j], j == 0 ? qprev : q[j - 1], vb[j]);
                    esc += (code == 0u);
                    hist_add(code, sh, a.hist);
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
            a.chunk_status[c] = 0ull;
        }
        __syncthreads();
    }
    for (int i = tid; i < kWin; i += kQuantThreads) {
        uint32_t v = sh[i];
        if (v) atomicAdd(&a.hist[kWinLo + i], v);
    }
}

void launch_quant(const CompressArgs* a, int k, void* stream) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    for (int i = 0; i < k; ++i) {
        uint32_t grid = umin32(a[i].n_chunks, (uint32_t)sms * 8u);
        if (grid == 0) grid = 1;
        quant_kernel<<<grid, kQuantThreads, 0, (cudaStream_t)stream>>>(a[i]);
    }
}

}  // namespace szg
