// sz_noalloc.cu -- sz_compress_noalloc: compression that allocates nothing.
//
// Some callers cannot let a library call cudaMalloc: an in-situ simulation
// that hands all device memory to its own pool, code running where a new
// allocation would synchronize the device, or a process under a hard memory
// cap.  This entry point runs the same four kernels as sz_compress (same
// stream, byte for byte), but every piece of scratch they need -- the array
// state, the code histogram, the codeword table, the per-chunk escape counts
// and look-back words, the codebook builder's work arrays and the error word
// -- lives in one file-scope static device array of fixed size.  That array
// exists on every GPU that loads the library, until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <mutex>
#include "sz_ctx.h"

using namespace szg;

namespace {

constexpr uint64_t kNoAllocMaxElems = 1ull << 26;    // largest n accepted (256 MB of float32)
constexpr uint64_t kNoAllocMaxChunks = 32768;        // 2^26 elements at the smallest chunk (2048)
constexpr size_t OFF_STATE = 0;
constexpr size_t OFF_ERR = 1024;
constexpr size_t OFF_HIST = 2048;
constexpr size_t OFF_ENC = OFF_HIST + sizeof(uint32_t) * kNumCodes;
constexpr size_t OFF_CESC = OFF_ENC + sizeof(uint32_t) * kNumCodes;
constexpr size_t OFF_CSTAT = OFF_CESC + sizeof(uint32_t) * kNoAllocMaxChunks;
constexpr size_t OFF_CB = OFF_CSTAT + sizeof(unsigned long long) * kNoAllocMaxChunks;
constexpr size_t kScratchBytes = OFF_CB + sizeof(uint32_t) * kCbScratchWords;   // about 5.9 MB
static_assert(sizeof(ArrayState) <= 1024, "state slot too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_ptr[kMaxDevices] = {};

// The device address of the array on the current device.  Host code only
// sees a stand-in for it, so the address comes from cudaGetSymbolAddress: on
// the first call per device (set-up) and again on every later call, so that a
// device whose context was reset and recreated -- which moves the array and
// zero-fills it -- gets its new address instead of a stale one.
sz_status device_scratch(int dev, uint8_t** out) {
    if (dev < 0 || dev >= kMaxDevices) return SZ_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    g_ptr[dev] = (uint8_t*)p;
    *out = g_ptr[dev];
    return SZ_OK;
}

// Arms the array state (range accumulators at their identities, everything
// else zero) and clears the error word, on the call's stream before its
// kernels, so that no call depends on what an earlier one left behind.
__global__ void __launch_bounds__(32) noalloc_arm_kernel(uint8_t* base) {
    uint32_t* w = reinterpret_cast<uint32_t*>(base + OFF_STATE);
    for (uint32_t i = threadIdx.x; i < sizeof(ArrayState) / 4; i += 32) w[i] = 0u;
    __syncwarp();
    if (threadIdx.x == 0) {
        ArrayState* st = reinterpret_cast<ArrayState*>(base + OFF_STATE);
        st->acc_min = 0xffffffffu;
        st->min_key = 0xffffffffu;
        *reinterpret_cast<uint32_t*>(base + OFF_ERR) = 0u;
    }
}

}  // namespace

extern "C" sz_status sz_compress_noalloc(const float* d_in, size_t n, double eb, sz_eb_kind kind, void* d_out,
                                         size_t out_cap, size_t* out_bytes, void* stream) {
    if (!out_bytes) return SZ_ERR_ARG;
    sz_status s = validate_compress(d_in, n, eb, kind, d_out);
    if (s != SZ_OK) return s;
    if ((uint64_t)n > kNoAllocMaxElems) return SZ_ERR_ARG;
    uint32_t C, G;
    if ((s = resolve_params(nullptr, n, &C, &G)) != SZ_OK) return s;
    const uint64_t nc = (n + C - 1) / C;
    if (nc > kNoAllocMaxChunks) return SZ_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    uint8_t* base = nullptr;
    if ((s = device_scratch(dev, &base)) != SZ_OK) return s;

    CompressArgs a;
    memset(&a, 0, sizeof(a));
    a.in = d_in;
    a.out = (uint8_t*)d_out;
    a.n = n;
    a.out_cap = out_cap;
    a.eb = eb;
    a.eb_kind = (int)kind;
    a.C = C;
    a.G = G;
    a.n_chunks = (uint32_t)nc;
    a.st = (ArrayState*)(base + OFF_STATE);
    a.hist = (uint32_t*)(base + OFF_HIST);
    a.enc = (uint32_t*)(base + OFF_ENC);
    a.chunk_esc = (uint32_t*)(base + OFF_CESC);
    a.chunk_status = (unsigned long long*)(base + OFF_CSTAT);
    a.cb_scratch = (uint32_t*)(base + OFF_CB);
    a.err = (uint32_t*)(base + OFF_ERR);

    cudaStream_t st = (cudaStream_t)stream;
    static_assert(sizeof(ArrayState) % 4 == 0, "state words");
    noalloc_arm_kernel<<<1, 32, 0, st>>>(base);
    launch_range(&a, 1, st);
    launch_quant(&a, 1, st);
    launch_codebook(&a, 1, st);
    launch_encode(&a, 1, st);
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    unsigned long long total = 0;
    uint32_t err = 0;
    if (cudaMemcpyAsync(&total, &a.st->total_bytes, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&err, a.err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    *out_bytes = (size_t)total;
    if (err & E_TIMEOUT) return SZ_ERR_TIMEOUT;
    if (err & E_CAPACITY) return SZ_ERR_CAPACITY;
    if (err) return SZ_ERR_CUDA;
    return SZ_OK;
}
