// k_quant.cu -- stand-alone launch of the quantize + histogram phase (a2-a4;
// body in sz_quant.cuh): persistent 256-thread blocks walk the chunks of one
// array with a block-private window of the histogram, flushed once at exit,
// each chunk's input staged into shared memory (one stage, so that four
// blocks fit on an SM).
#include "sz_quant.cuh"

namespace szg {

template <bool STORE, bool LCF = false>
__global__ void __launch_bounds__(kQuantThreads) quant_kernel(CompressArgs a) {
    __shared__ uint32_t sh[kWinWords];
    __shared__ uint32_t s_esc[kQuantThreads / 32];
    extern __shared__ float4 stage4[];
    const ArrayState* st = a.st;
    const LatticeParams P = st->P;
    if (P.raw || a.n == 0) return;
    hist_window_zero(sh);
    __syncthreads();
    if (((uintptr_t)a.in & 15u) == 0)
        quant_array_staged<STORE, LCF, 1>(a, P, blockIdx.x, gridDim.x, reinterpret_cast<float*>(stage4), sh, s_esc);
    else
        quant_array_global<STORE, LCF>(a, P, blockIdx.x, gridDim.x, sh, s_esc);
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
    // persistent grid: exactly the blocks that fit at once, for the stage of
    // the array's chunk size (two stages of C + 4 floats)
    // variants: 0 codes not stored, 1 stored, 2 stored with LCF prediction
    static int per_sm[3][4] = {};
    static const uint32_t kCs[4] = {2048u, 4096u, 8192u, 16384u};
    if (!per_sm[0][0]) {
        const int smax = (int)quant_stage_bytes(16384, 1);
        cudaFuncSetAttribute(quant_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(quant_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        cudaFuncSetAttribute(quant_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        for (int j = 0; j < 4; ++j) {
            const size_t sm = quant_stage_bytes(kCs[j], 1);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0][j], quant_kernel<false>, kQuantThreads, sm);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1][j], quant_kernel<true>, kQuantThreads, sm);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[2][j], quant_kernel<true, true>, kQuantThreads, sm);
            for (int v = 0; v < 3; ++v) if (per_sm[v][j] <= 0) per_sm[v][j] = 1;
        }
    }
    for (int i = 0; i < k; ++i) {
        // LCF needs the stored codes (its encoder does not recompute them)
        const int v = a[i].codes ? (a[i].pred == kPredLCF ? 2 : 1) : 0;
        const int j = a[i].C == 2048 ? 0 : a[i].C == 4096 ? 1 : a[i].C == 8192 ? 2 : 3;
        const size_t smem = quant_stage_bytes(a[i].C, 1);
        const uint32_t div = a[i].grid_div > 1 ? a[i].grid_div : 1u;
        uint32_t grid = umin32(a[i].n_chunks, (uint32_t)(sms * per_sm[v][j]) / div);
        if (grid == 0) grid = 1;
        if (v == 2)
            quant_kernel<true, true><<<grid, kQuantThreads, smem, (cudaStream_t)stream>>>(a[i]);
        else if (v)
            quant_kernel<true><<<grid, kQuantThreads, smem, (cudaStream_t)stream>>>(a[i]);
        else
            quant_kernel<false><<<grid, kQuantThreads, smem, (cudaStream_t)stream>>>(a[i]);
    }
}

}  // namespace szg
