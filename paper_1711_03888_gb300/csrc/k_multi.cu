// k_multi.cu -- the batched form's path for large arrays: each phase (a1
// range, a2-a4 quantize + histogram, a5 codebook, a6-a7 encode) is one launch
// over all large arrays of the batch, blockIdx.y selecting the array.  The
// bodies are the stand-alone kernels' (sz_range.cuh, sz_quant.cuh,
// sz_codebook.cuh, sz_encode.cuh), so every stream is byte-identical to
// sz_compress; the gain is that the arrays' single-block codebooks run side by
// side instead of one after another.  The four launches are kernel nodes of
// the batch's CUDA graph, on a branch parallel to the persistent kernel that
// takes the small arrays.
#include <cuda_runtime.h>
#include "sz_codebook.cuh"
#include "sz_encode.cuh"
#include "sz_quant.cuh"
#include "sz_range.cuh"

namespace szg {

namespace {

struct MultiArgs {
    const CompressArgs* args;   // device
    uint32_t first;             // array of blockIdx.y == 0
};

// the block's array, staged once in shared memory
__device__ __forceinline__ void stage_args(const MultiArgs& m, CompressArgs& sa) {
    if (threadIdx.x == 0) sa = m.args[m.first + blockIdx.y];
    __syncthreads();
}

__global__ void __launch_bounds__(256) range_multi_kernel(MultiArgs m) {
    __shared__ CompressArgs sa;
    stage_args(m, sa);
    range_body<256>(sa, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kQuantThreads) quant_multi_kernel(MultiArgs m) {
    __shared__ uint32_t sh[kWinWords];
    __shared__ uint32_t s_esc[kQuantThreads / 32];
    __shared__ CompressArgs sa;
    extern __shared__ float4 stage4[];
    stage_args(m, sa);
    const ArrayState* st = sa.st;
    const LatticeParams P = st->P;
    if (P.raw || sa.n == 0) return;
    hist_window_zero(sh);
    __syncthreads();
    if (((uintptr_t)sa.in & 15u) == 0)
        quant_array_staged<true>(sa, P, blockIdx.x, gridDim.x, reinterpret_cast<float*>(stage4), sh, s_esc);
    else
        quant_array_global<true>(sa, P, blockIdx.x, gridDim.x, sh, s_esc);
    hist_window_flush(sh, sa.hist);
}

__global__ void __launch_bounds__(kCbBlock) codebook_multi_kernel(MultiArgs m) {
    __shared__ CbSmem<kCbBlock> sm;
    __shared__ CompressArgs sa;
    extern __shared__ uint32_t fast[];
    stage_args(m, sa);
    codebook_body<kCbBlock>(sa, sm, fast, kCbFastSyms);
}

template <int C>
__global__ void __launch_bounds__(EncShape<C>::kThreads, EncShape<C>::kMinBlocks) encode_multi_kernel(MultiArgs m) {
    constexpr int NT = EncShape<C>::kThreads;
    extern __shared__ uint4 dyn_smem[];
    __shared__ EncSmem<NT> esm;
    __shared__ uint32_t s_c[2];
    __shared__ float s_prev;
    __shared__ CompressArgs sa;
    stage_args(m, sa);
    ArrayState* st = sa.st;
    if (sa.n == 0) return;
    if (st->raw) {
        const uint64_t words = (sa.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(sa, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    encode_array_pipelined<C, NT>(sa, reinterpret_cast<uint32_t*>(dyn_smem), esm, s_c, &s_prev);
}

constexpr int kEncSmem2048 = (int)enc_smem_bytes(2048);
constexpr int kEncSmem4096 = (int)enc_smem_bytes(4096);

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    return sms;
}

cudaError_t add_node(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps, void* func,
                     dim3 grid, dim3 block, size_t smem, MultiArgs* m) {
    cudaKernelNodeParams kp;
    memset(&kp, 0, sizeof(kp));
    void* kargs[] = {m};
    kp.func = func;
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = kargs;
    return cudaGraphAddKernelNode(node, g, deps, ndeps, &kp);
}

}  // namespace

int add_multi_compress_nodes(void* graph, void* dep, const CompressArgs* d_args, const MultiGroup* groups,
                             int ngroups) {
    if (ngroups <= 0) return 0;
    cudaGraph_t g = (cudaGraph_t)graph;
    cudaGraphNode_t d0 = (cudaGraphNode_t)dep;
    const uint32_t first = groups[0].first;
    uint32_t count = 0, max_nc = 1;
    for (int i = 0; i < ngroups; ++i) {
        count += groups[i].count;
        if (groups[i].max_chunks > max_nc) max_nc = groups[i].max_chunks;
    }
    static int per_sm = 0, enc_res[2] = {0, 0};
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(codebook_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbFastBytes);
        cudaFuncSetAttribute(quant_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)quant_stage_bytes(4096));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, quant_multi_kernel, kQuantThreads,
                                                      quant_stage_bytes(4096));
        if (per_sm <= 0) per_sm = 1;
        cudaFuncSetAttribute(encode_multi_kernel<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEncSmem2048);
        cudaFuncSetAttribute(encode_multi_kernel<4096>, cudaFuncAttributeMaxDynamicSharedMemorySize, kEncSmem4096);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&enc_res[0], encode_multi_kernel<2048>,
                                                      EncShape<2048>::kThreads, kEncSmem2048);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&enc_res[1], encode_multi_kernel<4096>,
                                                      EncShape<4096>::kThreads, kEncSmem4096);
        for (int j = 0; j < 2; ++j) enc_res[j] = (enc_res[j] > 0 ? enc_res[j] : 1) * sm_count();
        configured = true;
    }
    MultiArgs all{d_args, first};
    cudaGraphNode_t n_range, n_quant, n_cb;
    cudaError_t e;
    if ((e = add_node(g, &n_range, &d0, d0 ? 1 : 0, (void*)range_multi_kernel, dim3(kRangeBlocks, count), dim3(256), 0,
                      &all)) != cudaSuccess)
        return (int)e;
    const uint32_t qgrid = umin32(max_nc, (uint32_t)(sm_count() * per_sm));
    uint32_t maxC = 2048;
    for (int i = 0; i < ngroups; ++i) maxC = groups[i].C > maxC ? groups[i].C : maxC;
    if ((e = add_node(g, &n_quant, &n_range, 1, (void*)quant_multi_kernel, dim3(qgrid, count), dim3(kQuantThreads),
                      quant_stage_bytes(maxC), &all)) != cudaSuccess)
        return (int)e;
    if ((e = add_node(g, &n_cb, &n_quant, 1, (void*)codebook_multi_kernel, dim3(1, count), dim3(kCbBlock),
                      kCbFastBytes, &all)) != cudaSuccess)
        return (int)e;
    for (int i = 0; i < ngroups; ++i) {
        MultiArgs mg{d_args, groups[i].first};
        cudaGraphNode_t n_enc;
        // persistent encoders: the resident blocks shared out over the group's arrays
        const int j = groups[i].C == 2048 ? 0 : 1;
        const uint32_t per = umin32(groups[i].max_chunks ? groups[i].max_chunks : 1u,
                                    (uint32_t)(enc_res[j] / (int)groups[i].count > 0 ? enc_res[j] / (int)groups[i].count : 1));
        const dim3 grid(per, groups[i].count);
        if (groups[i].C == 2048)
            e = add_node(g, &n_enc, &n_cb, 1, (void*)encode_multi_kernel<2048>, grid,
                         dim3(EncShape<2048>::kThreads), kEncSmem2048, &mg);
        else if (groups[i].C == 4096)
            e = add_node(g, &n_enc, &n_cb, 1, (void*)encode_multi_kernel<4096>, grid,
                         dim3(EncShape<4096>::kThreads), kEncSmem4096, &mg);
        else
            return (int)cudaErrorInvalidValue;
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}

}  // namespace szg
