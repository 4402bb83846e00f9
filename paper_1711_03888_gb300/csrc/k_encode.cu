// k_encode.cu -- stand-alone launch of the encode phase (a6-a7; body in
// sz_encode.cuh): one block of C/32 threads per chunk, chunks taken in ticket
// order so the decoupled look-back only waits on running blocks.
#include "sz_encode.cuh"

namespace szg {

template <int NT, bool FROM_CODES>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 1 : 512 / NT)) encode_kernel(CompressArgs a) {
    extern __shared__ uint4 dyn_smem[];
    __shared__ EncSmem<NT> esm;
    __shared__ uint32_t s_c;
    ArrayState* st = a.st;
    if (st->raw) {
        const uint64_t words = (a.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(a, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    if (threadIdx.x == 0) s_c = atomicAdd(&st->ticket, 1u);
    __syncthreads();
    const uint32_t c = s_c;
    if (c >= a.n_chunks) return;
    encode_chunk<NT, 32, FROM_CODES>(a, c, reinterpret_cast<uint32_t*>(dyn_smem), esm);
}

template <int NT>
static void launch_encode_t(const CompressArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)NT * 32u * 4u;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(encode_kernel<NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(encode_kernel<NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured = true;
    }
    if (a.codes) encode_kernel<NT, true><<<a.n_chunks, NT, smem, s>>>(a);
    else encode_kernel<NT, false><<<a.n_chunks, NT, smem, s>>>(a);
}

void launch_encode(const CompressArgs* a, int k, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < k; ++i) {
        if (a[i].n == 0) continue;
        switch (a[i].C) {
            case 2048: launch_encode_t<64>(a[i], s); break;
            case 4096: launch_encode_t<128>(a[i], s); break;
            case 8192: launch_encode_t<256>(a[i], s); break;
            case 16384: launch_encode_t<512>(a[i], s); break;
            default: break;
        }
    }
}

}  // namespace szg
