// k_range.cu -- stand-alone launch of a1 (body in sz_range.cuh): a fixed grid
// of 256-thread blocks over one array.
#include "sz_range.cuh"

namespace szg {

__global__ void __launch_bounds__(256) range_kernel(CompressArgs a) { range_body<256>(a, blockIdx.x, gridDim.x); }

void launch_range(const CompressArgs* a, int k, void* stream) {
    for (int i = 0; i < k; ++i)
        range_kernel<<<kRangeBlocks, 256, 0, (cudaStream_t)stream>>>(a[i]);
}

}  // namespace szg
