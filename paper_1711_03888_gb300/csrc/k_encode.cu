// k_encode.cu -- stand-alone launch of the encode phase (a6-a7; body in
// sz_encode.cuh): one block of C/32 threads per chunk, chunks taken in ticket
// order so the decoupled look-back only waits on running blocks.
#include "sz_encode.cuh"

namespace szg {

template <int C, bool FROM_CODES>
__global__ void __launch_bounds__(EncShape<C>::kThreads, EncShape<C>::kMinBlocks) encode_kernel(CompressArgs a) {
    constexpr int NT = EncShape<C>::kThreads;
    extern __shared__ uint4 dyn_smem[];
    __shared__ EncSmem<NT> esm;
    __shared__ uint32_t s_c[2];
    __shared__ float s_prev;
    ArrayState* st = a.st;
    if (st->raw) {
        const uint64_t words = (a.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(a, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    uint32_t* smem = reinterpret_cast<uint32_t*>(dyn_smem);
    if (FROM_CODES) {
        encode_array_pipelined<C, NT>(a, smem, esm, s_c, &s_prev);
        return;
    }
    // codes recomputed from the input: one chunk per ticket
    for (;;) {
        if (threadIdx.x == 0) s_c[0] = atomicAdd(&st->ticket, 1u);
        __syncthreads();          // also: the last chunk's buffer is free
        const uint32_t c = s_c[0];
        __syncthreads();
        if (c >= a.n_chunks) return;
        encode_chunk<NT, EncShape<C>::kRun, false>(a, c, smem, esm);
    }
}

template <int C>
static void launch_encode_t(const CompressArgs& a, cudaStream_t s) {
    const size_t smem = enc_smem_bytes(C);
    constexpr int NT = EncShape<C>::kThreads;
    static int resident[2] = {0, 0};
    if (!resident[0]) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(encode_kernel<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(encode_kernel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int b0 = 0, b1 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b0, encode_kernel<C, false>, NT, smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, encode_kernel<C, true>, NT, smem);
        resident[0] = (b0 > 0 ? b0 : 1) * (sms > 0 ? sms : 148);
        resident[1] = (b1 > 0 ? b1 : 1) * (sms > 0 ? sms : 148);
    }
    // persistent: at most the resident blocks, each taking chunks by ticket
    const int v = a.codes ? 1 : 0;
    const uint32_t div = a.grid_div > 1 ? a.grid_div : 1u;
    uint32_t grid = umin32(a.n_chunks, (uint32_t)resident[v] / div);
    if (grid == 0) grid = 1;
    if (v) encode_kernel<C, true><<<grid, NT, smem, s>>>(a);
    else encode_kernel<C, false><<<grid, NT, smem, s>>>(a);
}

void launch_encode(const CompressArgs* a, int k, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < k; ++i) {
        if (a[i].n == 0) continue;
        switch (a[i].C) {
            case 2048: launch_encode_t<2048>(a[i], s); break;
            case 4096: launch_encode_t<4096>(a[i], s); break;
            case 8192: launch_encode_t<8192>(a[i], s); break;
            case 16384: launch_encode_t<16384>(a[i], s); break;
            default: break;
        }
    }
}

}  // namespace szg
