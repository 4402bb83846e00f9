// k_multi.cu -- the batched form's path for large arrays: each phase (a1
// range, a2-a4 quantize + histogram, a5 codebook, a6-a7 encode in two passes:
// chunk sizes, then packing) is one launch over all large arrays of the batch,
// blockIdx.y selecting the array.  The
// bodies are the stand-alone kernels' (sz_range.cuh, sz_quant.cuh,
// sz_codebook.cuh, sz_encode.cuh), so every stream is byte-identical to
// sz_compress; the gain is that the arrays' single-block codebooks run side by
// side instead of one after another.  multi_compress_launches describes the
// launches; the batch's CUDA graph takes them as kernel nodes on a branch
// parallel to the persistent kernel of the small arrays.
#include <cuda_runtime.h>
#include "../../include/sz_gb300.h"
#include "sz_codebook.cuh"
#include "sz_encode.cuh"
#include "sz_quant.cuh"
#include "sz_range.cuh"

namespace szg {

namespace {

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

// One input stage and four blocks per SM (64 registers, a few spills).
// Measured on GB300, six 2^27 arrays at rel eb 1e-3 / 1e-4 / 1e-5, quantize ms:
// 1.80 / 1.82 / 4.14 against 2.17 / 2.20 / 4.55 with two stages and no
// register bound (94 registers, two blocks per SM) and 1.87 / 1.88 / 4.48 with
// two stages at three blocks per SM.  Chunk-relative 32-bit offsets in the
// staged loop and the unaligned loop out of line cut the spills from 100 to
// 44 bytes: 1.60 / 1.62 / 3.91 against 1.71 / 1.73 / 3.99 ms (three blocks
// per SM without spills: 1.74 / 1.76 / 4.24).
#ifndef SZ_QMULTI_STAGES
#define SZ_QMULTI_STAGES 1
#endif
#ifndef SZ_QMULTI_MINB
#define SZ_QMULTI_MINB 4
#endif
// the unaligned-input loop, out of line so that its registers do not weigh
// on the staged loop's
__device__ __noinline__ void quant_multi_unaligned(const CompressArgs& a, uint32_t* sh, uint32_t* s_esc) {
    const LatticeParams P = a.st->P;
    quant_array_global<true>(a, P, blockIdx.x, gridDim.x, sh, s_esc);
}

// the histogram window after the input stage, in dynamic shared memory
// (0.02 ms less than a static window for six 2^27 arrays: fewer spills)
constexpr size_t kQWinBytes = 4u * kWinWords;
__global__ void __launch_bounds__(kQuantThreads, SZ_QMULTI_MINB) quant_multi_kernel(MultiArgs m) {
    __shared__ uint32_t s_esc[kQuantThreads / 32];
    __shared__ CompressArgs sa;
    extern __shared__ float4 stage4[];
    uint32_t* sh = reinterpret_cast<uint32_t*>(stage4);
    float* stagef = reinterpret_cast<float*>(stage4) + kWinWords;
    stage_args(m, sa);
    const ArrayState* st = sa.st;
    const LatticeParams P = st->P;
    if (P.raw || sa.n == 0) return;
    hist_window_zero(sh);
    __syncthreads();
    if (((uintptr_t)sa.in & 15u) == 0)
        quant_array_staged<true, false, SZ_QMULTI_STAGES>(sa, P, blockIdx.x, gridDim.x, stagef, sh, s_esc);
    else
        quant_multi_unaligned(sa, sh, s_esc);
    hist_window_flush(sh, sa.hist);
}

__global__ void __launch_bounds__(kCbBlock) codebook_multi_kernel(MultiArgs m) {
    __shared__ CbSmem<kCbBlock> sm;
    __shared__ CompressArgs sa;
    extern __shared__ uint32_t fast[];
    stage_args(m, sa);
    codebook_body<kCbBlock>(sa, sm, fast, kCbFastSyms, gridDim.x == 4u);
}

// pass 1 of the two-pass encoder over the group's arrays (gridDim.x blocks each)
template <int C>
__global__ void __launch_bounds__(kSizeThreads) encode_sizes_multi_kernel(MultiArgs m) {
    __shared__ EncSizesSmem sm;
    __shared__ CompressArgs sa;
    stage_args(m, sa);
    encode_sizes_body<C>(sa, gridDim.x, sm);
}

// pass 2: one warp per chunk at the offsets of pass 1
template <int C>
__global__ void __launch_bounds__(kPackWarps * 32, kPackMinBlocks) encode_pack_multi_kernel(MultiArgs m) {
    extern __shared__ uint4 pack_smem[];
    uint32_t* sm = reinterpret_cast<uint32_t*>(pack_smem);
    __shared__ CompressArgs sa;
    stage_args(m, sa);
    if (sa.n == 0) return;
    if (sa.st->raw) {
        const uint64_t words = (sa.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(sa, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    encode_pack_warp<C, false>(sa, sm + (threadIdx.x >> 5) * kRoundBufWords);
}

// one pass: persistent blocks with the chunks' look-back
#ifndef SZ_ENC_TWOPASS
#define SZ_ENC_TWOPASS 1
#endif
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
    encode_array_pipelined<C, NT, false, true>(sa, reinterpret_cast<uint32_t*>(dyn_smem), esm, s_c, &s_prev);
}

constexpr uint32_t kMultiC[4] = {2048u, 4096u, 8192u, 16384u};
const void* const kEncMulti[4] = {(const void*)encode_multi_kernel<2048>, (const void*)encode_multi_kernel<4096>,
                                  (const void*)encode_multi_kernel<8192>, (const void*)encode_multi_kernel<16384>};
constexpr int kEncThreads[4] = {EncShape<2048>::kThreads, EncShape<4096>::kThreads, EncShape<8192>::kThreads,
                                EncShape<16384>::kThreads};
const void* const kPackMulti[4] = {(const void*)encode_pack_multi_kernel<2048>,
                                   (const void*)encode_pack_multi_kernel<4096>,
                                   (const void*)encode_pack_multi_kernel<8192>,
                                   (const void*)encode_pack_multi_kernel<16384>};
const void* const kSizesMulti[4] = {(const void*)encode_sizes_multi_kernel<2048>,
                                    (const void*)encode_sizes_multi_kernel<4096>,
                                    (const void*)encode_sizes_multi_kernel<8192>,
                                    (const void*)encode_sizes_multi_kernel<16384>};

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

}  // namespace

int multi_compress_launches(const CompressArgs* d_args, const MultiGroup* groups, int ngroups, KernelLaunch* out,
                            int max_out) {
    if (ngroups <= 0) return 0;
    if (max_out < 3 + 2 * ngroups) return -1;
    const uint32_t first = groups[0].first;
    uint32_t count = 0, max_nc = 1, maxC = 2048;
    for (int i = 0; i < ngroups; ++i) {
        count += groups[i].count;
        if (groups[i].max_chunks > max_nc) max_nc = groups[i].max_chunks;
        if (groups[i].C > maxC) maxC = groups[i].C;
    }
    static int quant_res[4] = {0, 0, 0, 0}, enc_res[4] = {0, 0, 0, 0}, size_res = 0, pack_res = 0;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(codebook_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbFastBytes);
        cudaFuncSetAttribute(quant_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(quant_stage_bytes(16384, SZ_QMULTI_STAGES) + kQWinBytes));
        for (int j = 0; j < 4; ++j) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&quant_res[j], quant_multi_kernel, kQuantThreads,
                                                          quant_stage_bytes(kMultiC[j], SZ_QMULTI_STAGES) + kQWinBytes);
            quant_res[j] = (quant_res[j] > 0 ? quant_res[j] : 1) * sm_count();
        }
        for (int j = 0; j < 4; ++j) {
            const int sm = (int)enc_smem_bytes((int)kMultiC[j]);
            cudaFuncSetAttribute(kEncMulti[j], cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&enc_res[j], kEncMulti[j], kEncThreads[j], sm);
            enc_res[j] = (enc_res[j] > 0 ? enc_res[j] : 1) * sm_count();
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&size_res, kSizesMulti[1], kSizeThreads, 0);
        size_res = (size_res > 0 ? size_res : 1) * sm_count();
        for (int j = 0; j < 4; ++j)
            cudaFuncSetAttribute(kPackMulti[j], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pack_smem_bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pack_res, kPackMulti[1], kPackWarps * 32, pack_smem_bytes());
        pack_res = (pack_res > 0 ? pack_res : 1) * sm_count();
        configured = true;
    }
    auto set = [](KernelLaunch& L, const void* f, uint32_t gx, uint32_t gy, uint32_t bx, size_t smem, int phase,
                  const CompressArgs* args, uint32_t first) {
        L.func = f;
        L.grid[0] = gx; L.grid[1] = gy; L.grid[2] = 1;
        L.block[0] = bx; L.block[1] = 1; L.block[2] = 1;
        L.smem = smem;
        L.phase = phase;
        L.args = MultiArgs{args, first};
    };
    int k = 0;
    set(out[k++], (const void*)range_multi_kernel, kRangeBlocks, count, 256, 0, SZ_PHASE_RANGE, d_args, first);
    const int jq = maxC == 2048 ? 0 : maxC == 4096 ? 1 : maxC == 8192 ? 2 : 3;
    set(out[k++], (const void*)quant_multi_kernel, umin32(max_nc, (uint32_t)quant_res[jq]), count,
        kQuantThreads, quant_stage_bytes(maxC, SZ_QMULTI_STAGES) + kQWinBytes, SZ_PHASE_QUANT, d_args, first);
    set(out[k++], (const void*)codebook_multi_kernel, kCbBlocks, count, kCbBlock, kCbFastBytes, SZ_PHASE_CODEBOOK, d_args,
        first);
    for (int i = 0; i < ngroups; ++i) {
        // persistent encoders: the resident blocks shared out over the group's arrays
        int j = -1;
        for (int t = 0; t < 4; ++t)
            if (groups[i].C == kMultiC[t]) j = t;
        if (j < 0) return -1;
        const uint32_t mc = groups[i].max_chunks ? groups[i].max_chunks : 1u;
        const int sshare = size_res / (int)groups[i].count;
        if (k >= max_out) return -1;
        if (SZ_ENC_TWOPASS)
            set(out[k++], kSizesMulti[j], umin32(mc, (uint32_t)(sshare > 0 ? sshare : 1)), groups[i].count,
                kSizeThreads, 0, SZ_PHASE_ENCODE_SIZES, d_args, groups[i].first);
        if (k >= max_out) return -1;
        if (SZ_ENC_TWOPASS) {
            const int pshare = pack_res / (int)groups[i].count;
            set(out[k++], kPackMulti[j], umin32((mc + kPackWarps - 1) / kPackWarps, (uint32_t)(pshare > 0 ? pshare : 1)),
                groups[i].count, kPackWarps * 32, pack_smem_bytes(), SZ_PHASE_ENCODE, d_args, groups[i].first);
        } else {
            const int share = enc_res[j] / (int)groups[i].count;
            const uint32_t per = umin32(mc, (uint32_t)(share > 0 ? share : 1));
            set(out[k++], kEncMulti[j], per, groups[i].count, kEncThreads[j], enc_smem_bytes((int)kMultiC[j]),
                SZ_PHASE_ENCODE, d_args, groups[i].first);
        }
    }
    return k;
}

}  // namespace szg
