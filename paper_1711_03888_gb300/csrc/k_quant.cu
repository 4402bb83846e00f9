// k_quant.cu -- stand-alone launch of the quantize + histogram phase (a2-a4;
// body in sz_quant.cuh): persistent 256-thread blocks walk the chunks of one
// array with a block-private window of the histogram, flushed once at exit.
#include "sz_quant.cuh"

namespace szg {

template <bool STORE>
__global__ void __launch_bounds__(kQuantThreads) quant_kernel(CompressArgs a) {
    __shared__ uint32_t sh[kWin];
    __shared__ uint32_t s_esc[kQuantThreads / 32];
    const ArrayState* st = a.st;
    const LatticeParams P = st->P;
    if (P.raw || a.n == 0) return;
    hist_window_zero(sh);
    __syncthreads();
    for (uint32_t c = blockIdx.x; c < a.n_chunks; c += gridDim.x) quant_chunk<STORE>(a, P, c, sh, s_esc);
    hist_window_flush(sh, a.hist);
}

void launch_quant(const CompressArgs* a, int k, void* stream) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    // persistent grid: exactly the blocks that fit at once
    static int per_sm[2] = {0, 0};
    if (!per_sm[0]) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], quant_kernel<false>, kQuantThreads, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], quant_kernel<true>, kQuantThreads, 0);
        for (int j = 0; j < 2; ++j) if (per_sm[j] <= 0) per_sm[j] = 1;
    }
    for (int i = 0; i < k; ++i) {
        const int v = a[i].codes ? 1 : 0;
        const uint32_t div = a[i].grid_div > 1 ? a[i].grid_div : 1u;
        uint32_t grid = umin32(a[i].n_chunks, umin32((uint32_t)(sms * per_sm[v]) / div, (uint32_t)(sms * per_sm[v])));
        if (grid == 0) grid = 1;
        if (v)
            quant_kernel<true><<<grid, kQuantThreads, 0, (cudaStream_t)stream>>>(a[i]);
        else
            quant_kernel<false><<<grid, kQuantThreads, 0, (cudaStream_t)stream>>>(a[i]);
    }
}

}  // namespace szg
