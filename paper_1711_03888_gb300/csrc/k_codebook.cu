// k_codebook.cu -- stand-alone launch of the codebook phase (body in sz_codebook.cuh).
#include "sz_codebook.cuh"

namespace szg {

__global__ void __launch_bounds__(kCbBlock) codebook_kernel(CompressArgs a) {
    __shared__ CbSmem<kCbBlock> sm;
    extern __shared__ uint32_t fast[];
    codebook_body<kCbBlock>(a, sm, fast, kCbFastSyms, gridDim.x == 4u);
}

void launch_codebook(const CompressArgs* a, int k, void* stream) {
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(codebook_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbFastBytes);
        configured = true;
    }
    for (int i = 0; i < k; ++i) codebook_kernel<<<kCbBlocks, kCbBlock, kCbFastBytes, (cudaStream_t)stream>>>(a[i]);
}

}  // namespace szg
