// k_codebook.cu -- stand-alone launch of the codebook phase (body in sz_codebook.cuh).
#include "sz_codebook.cuh"

namespace szg {

__global__ void __launch_bounds__(kCbBlock) codebook_kernel(CompressArgs a) {
    __shared__ CbSmem<kCbBlock> sm;
    codebook_body<kCbBlock>(a, sm);
}

void launch_codebook(const CompressArgs* a, int k, void* stream) {
    for (int i = 0; i < k; ++i) codebook_kernel<<<1, kCbBlock, 0, (cudaStream_t)stream>>>(a[i]);
}

}  // namespace szg
