// k_batch.cu -- a15: the batched form.  One persistent launch compresses k
// independent arrays (the per-rank fields of a snapshot; Sec. V compresses
// every in-memory array independently).
//
// The work list holds every array's items in dependency order:
//   range tiles (plan.range_tile elements) -> quantize groups (plan.quant_group
//   chunks) -> one codebook per array -> encode chunks
// Blocks of 256 threads take items from one atomic counter.  Before running
// an item a block waits (bounded) on the per-array counters its phase needs.
// Every item a block can wait on was taken earlier by a running block, whose
// own waits only point further back, so the launch cannot deadlock.  Small
// arrays finish their codebook and encoding while large ones are still
// being quantized; per-array fixed costs (the single-block codebook) overlap
// across arrays instead of adding up.  Each array's stream is byte-identical
// to sz_compress on that array.
#include "sz_codebook.cuh"
#include "sz_encode.cuh"
#include "sz_quant.cuh"

namespace szg {

constexpr int kBatchThreads = 256;
// a quantize item flushes its histogram window once: its elements must fit
// the window's 16-bit counters, so quant_group * C <= 65535 (the host checks)
constexpr uint32_t kWaitSpins = 1u << 24;

union BatchSmem {
    struct {
        uint32_t win[kWinWords];
        uint32_t esc[kQuantThreads / 32];
    } q;
    CbSmem<kBatchThreads> cb;
    struct {
        uint32_t buf[kBatchThreads * 16];    // C <= 4096 words
        EncSmem<kBatchThreads> esm;
    } e;
    struct {
        uint32_t kmin[8], kmax[8], any[8];
    } r;
};

struct BatchCtl {
    uint32_t item;        // current item (broadcast)
    uint32_t ok;          // dependencies satisfied
};

// bounded wait by thread 0 for *flag >= target; false (and E_TIMEOUT) on expiry
__device__ __forceinline__ bool wait_at_least(const uint32_t* flag, uint32_t target, uint32_t* err) {
    uint32_t spins = 0;
    for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= target) return true;
        if (++spins > kWaitSpins) {
            atomicOr(err, E_TIMEOUT);
            return false;
        }
        __nanosleep(128);
    }
}

__device__ __forceinline__ void signal_add(uint32_t* p, uint32_t v) {
    __threadfence();
    atomicAdd(p, v);
}

// last index i with off[i] <= x, for a non-decreasing off[0..k]
__device__ __forceinline__ uint32_t find_array(const uint32_t* off, uint32_t k, uint32_t x) {
    uint32_t lo = 0, hi = k;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
    }
    return lo;
}

__device__ void batch_range_tile(const CompressArgs& a, BatchCounters* cnt, uint32_t t, uint32_t ntiles,
                                 uint32_t tile, BatchSmem& sm) {
    const int tid = threadIdx.x;
    // share of the histogram to clear
    const uint32_t per = (kNumCodes + ntiles - 1) / ntiles;
    for (uint32_t i = t * per + tid; i < umin32((t + 1) * per, kNumCodes); i += kBatchThreads) a.hist[i] = 0u;
    uint32_t kmin = 0xffffffffu, kmax = 0u, any = 0u;
    if (a.eb_kind == 1) {
        const uint64_t b = (uint64_t)t * tile, e = umin64(a.n, b + tile);
        for (uint64_t i = b + tid; i < e; i += kBatchThreads) {
            float x = __ldg(a.in + i);
            if (finite_f(x)) {
                uint32_t k = float_key(x);
                kmin = min(kmin, k);
                kmax = max(kmax, k);
                any = 1u;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        any |= __shfl_xor_sync(0xffffffffu, any, o);
    }
    if ((tid & 31) == 0) { sm.r.kmin[tid >> 5] = kmin; sm.r.kmax[tid >> 5] = kmax; sm.r.any[tid >> 5] = any; }
    __threadfence();          // this thread's histogram clears, before the tile is counted
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < kBatchThreads / 32; ++w) {
            kmin = min(kmin, sm.r.kmin[w]);
            kmax = max(kmax, sm.r.kmax[w]);
            any |= sm.r.any[w];
        }
        ArrayState* st = a.st;
        if (any) {
            atomicMin(&st->acc_min, kmin);
            atomicMax(&st->acc_max, kmax);
            atomicOr(&st->acc_any, 1u);
        }
        __threadfence();
        if (atomicAdd(&cnt->range_done, 1u) == ntiles - 1) {
            __threadfence();
            const uint32_t kmin2 = atomicExch(&st->acc_min, 0xffffffffu);
            const uint32_t kmax2 = atomicExch(&st->acc_max, 0u);
            const uint32_t any2 = atomicExch(&st->acc_any, 0u);
            st->min_key = kmin2;
            st->max_key = kmax2;
            st->any_finite = any2;
            st->P = make_params(range_eb_abs(a.eb, a.eb_kind, kmin2, kmax2, any2));
            signal_add(&cnt->range_ready, 1u);
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kBatchThreads) batch_compress_kernel(BatchPlan plan) {
    extern __shared__ uint4 dyn_smem[];
    BatchSmem& sm = *reinterpret_cast<BatchSmem*>(dyn_smem);
    __shared__ BatchCtl ctl;
    const int tid = threadIdx.x;
    const uint32_t k = plan.k;
    const uint32_t* off = plan.item_off;       // 4 phases x (k + 1)
    const uint32_t p1 = off[k], p2 = off[(k + 1) + k], p3 = off[2 * (k + 1) + k], p4 = off[3 * (k + 1) + k];
    for (;;) {
        if (tid == 0) ctl.item = atomicAdd(plan.next, 1u);
        __syncthreads();
        const uint32_t item = ctl.item;
        __syncthreads();
        if (item >= p4) return;
        const int phase = item < p1 ? 0 : (item < p2 ? 1 : (item < p3 ? 2 : 3));
        const uint32_t* po = off + phase * (k + 1);
        const uint32_t arr = find_array(po, k, item);
        const uint32_t idx = item - po[arr];
        const CompressArgs& a = plan.args[arr];
        BatchCounters* cnt = plan.cnt + arr;
        // ---- dependencies ---------------------------------------------------------
        if (tid == 0) {
            bool ok = true;
            if (phase >= 1) ok = wait_at_least(&cnt->range_ready, 1u, plan.err);
            if (ok && phase >= 2) ok = wait_at_least(&cnt->quant_done, plan.quant_groups[arr], plan.err);
            if (ok && phase == 3) ok = wait_at_least(&cnt->cb_ready, 1u, plan.err);
            ctl.ok = ok;
        }
        __syncthreads();
        if (!ctl.ok) continue;
        // ---- the item ---------------------------------------------------------------
        if (phase == 0) {
            batch_range_tile(a, cnt, idx, plan.range_tiles[arr], plan.range_tile, sm);
        } else if (phase == 1) {
            const ArrayState* st = a.st;
            const LatticeParams P = st->P;
            if (!P.raw && a.n) {
                hist_window_zero(sm.q.win);
                __syncthreads();
                const uint32_t g = plan.quant_group;
                const uint32_t c1 = umin32((idx + 1) * g, a.n_chunks);
                for (uint32_t c = idx * g; c < c1; ++c) quant_chunk<true>(a, P, c, sm.q.win, sm.q.esc);
                hist_window_flush(sm.q.win, a.hist);
            }
            __threadfence();      // codes, escape counts and histogram before the group is counted
            __syncthreads();
            if (tid == 0) signal_add(&cnt->quant_done, 1u);
        } else if (phase == 2) {
            codebook_body<kBatchThreads>(a, sm.cb);
            __threadfence();      // codeword table, layout and header before the encoders start
            __syncthreads();
            if (tid == 0) signal_add(&cnt->cb_ready, 1u);
        } else {
            if (a.st->raw) {
                const uint64_t words = (a.n + 3u) & ~(uint64_t)3u;
                const uint64_t wb = (uint64_t)idx * a.C, we = umin64(words, wb + a.C);
                raw_copy_words(a, wb, we, tid, kBatchThreads);
            } else if (a.C == 4096) {
                encode_chunk<kBatchThreads, 16, true>(a, idx, sm.e.buf, sm.e.esm);
            } else {
                encode_chunk<kBatchThreads, 8, true>(a, idx, sm.e.buf, sm.e.esm);
            }
        }
        __syncthreads();
    }
}

void batch_compress_config(void** func, unsigned* grid, unsigned* block, size_t* smem) {
    static int g = 0;
    const size_t sm = sizeof(BatchSmem);
    if (!g) {
        cudaFuncSetAttribute(batch_compress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_compress_kernel, kBatchThreads, sm);
        g = (sms > 0 ? sms : 148) * (per > 0 ? per : 1);
    }
    *func = (void*)batch_compress_kernel;
    *grid = (unsigned)g;
    *block = kBatchThreads;
    *smem = sm;
}

void launch_batch_compress(const BatchPlan& plan, void* stream) {
    void* f;
    unsigned grid, block;
    size_t smem;
    batch_compress_config(&f, &grid, &block, &smem);
    batch_compress_kernel<<<grid, block, smem, (cudaStream_t)stream>>>(plan);
}

}  // namespace szg
