// k_encode.cu -- stand-alone launch of the encode phase (a6-a7; bodies in
// sz_encode.cuh).  Arrays of kTwoPassChunks chunks or more take the two-pass
// encoder: pass 1 (encode_sizes_kernel) writes the chunk-word table, pass 2
// (encode_kernel, LOOKBACK = false) packs every chunk at its offset with no
// waits.  Smaller arrays, and codes recomputed from the input, take one pass:
// persistent blocks take chunks in ticket order and find their offsets by the
// decoupled look-back, which only waits on running blocks.
#include "sz_encode.cuh"

namespace szg {

#ifndef SZ_ENC_TWOPASS
#define SZ_ENC_TWOPASS 1
#endif
constexpr uint32_t kTwoPassChunks = SZ_ENC_TWOPASS ? 64u : 0xffffffffu;

template <int C>
__global__ void __launch_bounds__(kSizeThreads) encode_sizes_kernel(CompressArgs a, uint32_t nblocks) {
    __shared__ EncSizesSmem sm;
    encode_sizes_body<C>(a, nblocks, sm);
}

template <int C, bool LCF>
__global__ void __launch_bounds__(kPackWarps * 32, kPackMinBlocks) encode_pack_kernel(CompressArgs a) {
    extern __shared__ uint4 pack_smem[];
    uint32_t* sm = reinterpret_cast<uint32_t*>(pack_smem);
    if (a.st->raw) {
        const uint64_t words = (a.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(a, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    encode_pack_warp<C, LCF>(a, sm + (threadIdx.x >> 5) * kRoundBufWords);
}

template <int C, bool FROM_CODES, bool LCF = false, bool LOOKBACK = true>
__global__ void __launch_bounds__(EncShape<C>::kThreads, EncShape<C>::kMinBlocks) encode_kernel(CompressArgs a) {
    static_assert(FROM_CODES || !LCF, "LCF encodes the stored codes");
    constexpr int NT = EncShape<C>::kThreads;
    extern __shared__ uint4 dyn_smem[];
    __shared__ EncSmem<NT> esm;
    __shared__ uint32_t s_c[2];
    __shared__ float s_prev[2];
    ArrayState* st = a.st;
    if (st->raw) {
        const uint64_t words = (a.n + 3u) & ~(uint64_t)3u;
        raw_copy_words(a, 0, words, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
        return;
    }
    uint32_t* smem = reinterpret_cast<uint32_t*>(dyn_smem);
    if constexpr (FROM_CODES) {
        encode_array_pipelined<C, NT, LCF, LOOKBACK>(a, smem, esm, s_c, s_prev);
    } else {
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
}

template <int C>
static void launch_encode_t(const CompressArgs& a, cudaStream_t s) {
    const size_t smem = enc_smem_bytes(C);
    constexpr int NT = EncShape<C>::kThreads;
    // variants: 0 codes recomputed, 1 stored codes, 2 stored codes with LCF; then
    // 3 and 4: the packing pass of the two-pass encoder (LV, LCF)
    static int resident[5] = {0, 0, 0, 0, 0};
    static int sms = 0, size_res = 0, pack_res[2] = {0, 0};
    if (!resident[0]) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
        const void* f[5] = {(const void*)encode_kernel<C, false>, (const void*)encode_kernel<C, true>,
                            (const void*)encode_kernel<C, true, true>, (const void*)encode_kernel<C, true, false, false>,
                            (const void*)encode_kernel<C, true, true, false>};
        for (int v = 0; v < 5; ++v) {
            cudaFuncSetAttribute(f[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f[v], NT, smem);
            resident[v] = (b > 0 ? b : 1) * sms;
        }
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, encode_sizes_kernel<C>, kSizeThreads, 0);
        size_res = (b > 0 ? b : 1) * sms;
        cudaFuncSetAttribute(encode_pack_kernel<C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pack_smem_bytes());
        cudaFuncSetAttribute(encode_pack_kernel<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pack_smem_bytes());
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, encode_pack_kernel<C, false>, kPackWarps * 32,
                                                      pack_smem_bytes());
        pack_res[0] = (b > 0 ? b : 1) * sms;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, encode_pack_kernel<C, true>, kPackWarps * 32,
                                                      pack_smem_bytes());
        pack_res[1] = (b > 0 ? b : 1) * sms;
    }
    // persistent: at most the resident blocks, each taking chunks by ticket
    // (the quantizer stores the codes whenever the prediction is LCF)
    int v = a.codes ? (a.pred == kPredLCF ? 2 : 1) : 0;
    const uint32_t div = a.grid_div > 1 ? a.grid_div : 1u;
    if (v && a.n_chunks >= kTwoPassChunks) {
        const uint32_t nb = umin32(a.n_chunks, umax32(1u, (uint32_t)size_res / div));
        encode_sizes_kernel<C><<<nb, kSizeThreads, 0, s>>>(a, nb);
        const int l = v == 2 ? 1 : 0;
        const uint32_t np = umin32((a.n_chunks + kPackWarps - 1) / kPackWarps, umax32(1u, (uint32_t)pack_res[l] / div));
        if (l) encode_pack_kernel<C, true><<<np, kPackWarps * 32, pack_smem_bytes(), s>>>(a);
        else encode_pack_kernel<C, false><<<np, kPackWarps * 32, pack_smem_bytes(), s>>>(a);
        return;
    }
    uint32_t grid = umin32(a.n_chunks, (uint32_t)resident[v] / div);
    if (grid == 0) grid = 1;
    switch (v) {
        case 0: encode_kernel<C, false><<<grid, NT, smem, s>>>(a); break;
        case 1: encode_kernel<C, true><<<grid, NT, smem, s>>>(a); break;
        case 2: encode_kernel<C, true, true><<<grid, NT, smem, s>>>(a); break;
        case 3: encode_kernel<C, true, false, false><<<grid, NT, smem, s>>>(a); break;
        default: encode_kernel<C, true, true, false><<<grid, NT, smem, s>>>(a); break;
    }
}

// The timeout path of the look-back wait: one warp waits, as the encoder of
// chunk 1 would, on chunk 0's status word, which nothing publishes.  After
// `spins` polls the wait gives up and the kernel latches E_TIMEOUT.
__global__ void __launch_bounds__(32) wait_timeout_kernel(unsigned long long* status, uint32_t* err, uint32_t spins) {
    if (threadIdx.x == 0) st_status(&status[0], 0ull);
    __syncwarp();
    unsigned long long excl = 0;
    const bool ok = lookback_prefix(status, 1, spins, &excl);
    if (threadIdx.x == 0 && !ok) raise_err(err, E_TIMEOUT);
}

void launch_wait_timeout(unsigned long long* status, uint32_t* err, uint32_t spins, void* stream) {
    wait_timeout_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(status, err, spins);
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
