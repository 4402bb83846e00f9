// sz_batch.cu -- many arrays per call (a15).
//
// Compression: one CUDA graph per batch shape, replayed on every call.  Its
// nodes: the plan copy and a counter reset, then two parallel branches --
//   small arrays (< 2^22 elements): one persistent launch (k_batch.cu) over
//     every array's range, quantize, codebook and encode items;
//   large arrays: one launch per phase over all of them (k_multi.cu).
// The context keeps a batch pool with each array's own state, histogram,
// codeword table, codebook scratch and per-chunk tables, sliced by that
// array's size.  Each stream is byte-identical to sz_compress on the same
// array.  Arrays whose chunk size is above 4096 (set explicitly through
// params) go through the per-array path instead.
// Decompression (k > 1): one setup launch (a block per stream), a scan of the
// streams' decode units, and one decode launch whose blocks take contiguous
// ranges of all streams' chunks (k_decode.cu).
#include <algorithm>
#include <string.h>
#include <vector>
#include "sz_ctx.h"

namespace szg {

namespace {

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

sz_status pool_reserve(sz_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->batch_bytes) return SZ_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) return SZ_ERR_CUDA;
    if (ctx->batch_pool) cudaFree(ctx->batch_pool);
    ctx->batch_pool = nullptr;
    ctx->batch_bytes = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
    ctx->batch_pool = (uint8_t*)p;
    ctx->batch_bytes = bytes;
    ctx->batch_states_armed = 0;
    return SZ_OK;
}

}  // namespace

sz_status batch_compress(sz_ctx* ctx, int k, const float* const* d_in, const size_t* n, const double* eb,
                         sz_eb_kind kind, const sz_params* params, void* const* d_out, const size_t* out_cap,
                         size_t* out_bytes, cudaStream_t s) {
    cudaSetDevice(ctx->device);
    std::vector<uint32_t> Cs(k), Gs(k);
    std::vector<int> batched;
    const bool lcf = params_pred(params) == kPredLCF;
    for (int i = 0; i < k; ++i) {
        sz_status st = validate_compress(d_in[i], n[i], eb[i], kind, d_out[i]);
        if (st != SZ_OK) return st;
        if ((st = resolve_params(params, n[i], &Cs[i], &Gs[i])) != SZ_OK) return st;
        if (Cs[i] <= 4096 && !lcf) batched.push_back(i);
    }
    // arrays with large explicit chunks or LCF prediction: the per-array path
    for (int i = 0; i < k; ++i) {
        if (Cs[i] <= 4096 && !lcf) continue;
        sz_status st = sz_compress(ctx, d_in[i], n[i], eb[i], kind, params, d_out[i], out_cap[i],
                                   out_bytes ? &out_bytes[i] : nullptr, s);
        if (st != SZ_OK) return st;
    }
    const uint32_t kb = (uint32_t)batched.size();
    if (kb == 0) return SZ_OK;
    // Small arrays first (the persistent kernel's), then the others grouped by
    // C (the per-phase launches').  A few small arrays are latency-bound by
    // their codebooks, so they take the per-phase launches too (1024-thread
    // codebooks side by side); many small arrays keep the persistent kernel,
    // where their codebook items overlap the other arrays' work.
    uint32_t ks = 0;
    {
        std::vector<int> small, large;
        for (int i : batched) (n[i] < kBatchLargeElems ? small : large).push_back(i);
        if (small.size() <= kBatchFewSmall) {
            large.insert(large.begin(), small.begin(), small.end());
            small.clear();
        }
        std::stable_sort(large.begin(), large.end(), [&](int x, int y) { return Cs[x] < Cs[y]; });
        ks = (uint32_t)small.size();
        batched = small;
        batched.insert(batched.end(), large.begin(), large.end());
    }
    std::vector<MultiGroup> groups;
    for (uint32_t j = ks; j < kb; ++j) {
        const int i = batched[j];
        const uint32_t nc = (uint32_t)((n[i] + Cs[i] - 1) / Cs[i]);
        if (groups.empty() || groups.back().C != Cs[i]) groups.push_back(MultiGroup{j, 0u, Cs[i], 0u});
        groups.back().count++;
        if (nc > groups.back().max_chunks) groups.back().max_chunks = nc;
    }

    // ---- pool layout: plan | counters | states | per-array buffers ------------------
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += align256(b); return o; };
    const size_t o_args = take(sizeof(CompressArgs) * kb);
    const size_t o_tiles = take(sizeof(uint32_t) * (ks + 1));
    const size_t o_groups = take(sizeof(uint32_t) * (ks + 1));
    const size_t o_off = take(sizeof(uint32_t) * 4 * (ks + 1));
    const size_t plan_bytes = bytes;
    const size_t cnt_bytes = sizeof(BatchCounters) * ks + 256;
    const size_t o_cnt = take(cnt_bytes);
    const size_t o_state = take(sizeof(ArrayState) * kb);
    std::vector<size_t> o_hist(kb), o_enc(kb), o_cb(kb), o_cesc(kb), o_cst(kb), o_codes(kb);
    for (uint32_t j = 0; j < kb; ++j) {
        const int i = batched[j];
        const uint64_t nc = (n[i] + Cs[i] - 1) / Cs[i];
        o_hist[j] = take(sizeof(uint32_t) * kNumCodes);
        o_enc[j] = take(sizeof(uint32_t) * kNumCodes);
        o_cb[j] = take(sizeof(uint32_t) * kCbScratchWords);
        o_cesc[j] = take(sizeof(uint32_t) * (nc + 1));
        o_cst[j] = take(sizeof(unsigned long long) * (nc + 1));
        o_codes[j] = take(sizeof(uint16_t) * (nc * Cs[i] + 8));
    }
    sz_status st = pool_reserve(ctx, bytes);
    if (st != SZ_OK) return st;
    uint8_t* base = ctx->batch_pool;

    // ---- plan -------------------------------------------------------------------
    std::vector<CompressArgs> args(kb);
    std::vector<uint32_t> tiles(ks + 1), qgroups(ks + 1), off(4 * (ks + 1));
    uint32_t item = 0;
    for (int ph = 0; ph < 4; ++ph) {
        for (uint32_t j = 0; j < ks; ++j) {
            const int i = batched[j];
            const uint64_t nc = (n[i] + Cs[i] - 1) / Cs[i];
            off[ph * (ks + 1) + j] = item;
            uint32_t cnt;
            if (ph == 0) cnt = tiles[j] = (uint32_t)((n[i] + kRangeTile - 1) / kRangeTile) + (n[i] == 0 ? 1u : 0u);
            else if (ph == 1) cnt = qgroups[j] = (uint32_t)((nc + kQuantGroup - 1) / kQuantGroup);
            else if (ph == 2) cnt = 1;
            else cnt = (uint32_t)nc;
            item += cnt;
        }
        off[ph * (ks + 1) + ks] = item;
    }
    uint64_t key = 1469598103934665603ull;      // FNV-1a over everything the graph bakes in
    auto mix = [&](const void* p, size_t b) {
        const uint8_t* c = (const uint8_t*)p;
        for (size_t t = 0; t < b; ++t) key = (key ^ c[t]) * 1099511628211ull;
    };
    mix(&base, sizeof(base));
    mix(&bytes, sizeof(bytes));
    for (uint32_t j = 0; j < kb; ++j) {
        const int i = batched[j];
        CompressArgs& a = args[j];
        memset(&a, 0, sizeof(a));
        a.in = d_in[i];
        a.out = (uint8_t*)d_out[i];
        a.n = n[i];
        a.out_cap = out_cap[i];
        a.eb = eb[i];
        a.eb_kind = (int)kind;
        a.C = Cs[i];
        a.G = Gs[i];
        a.n_chunks = (uint32_t)((n[i] + Cs[i] - 1) / Cs[i]);
        a.st = (ArrayState*)(base + o_state) + j;
        a.hist = (uint32_t*)(base + o_hist[j]);
        a.enc = (uint32_t*)(base + o_enc[j]);
        a.cb_scratch = (uint32_t*)(base + o_cb[j]);
        a.chunk_esc = (uint32_t*)(base + o_cesc[j]);
        a.chunk_status = (unsigned long long*)(base + o_cst[j]);
        a.codes = (uint16_t*)(base + o_codes[j]);
        a.err = ctx->d_err;
        mix(&a, sizeof(a));
    }

    if (key != ctx->bg_key || !ctx->bg_exec) {
        // a new batch: wait for the previous graph before reusing its staging
        if (ctx->bg_done && cudaEventSynchronize(ctx->bg_done) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
        if (!ctx->bg_done && cudaEventCreateWithFlags(&ctx->bg_done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return SZ_ERR_CUDA;
        }
        if (plan_bytes > ctx->batch_host_bytes) {
            if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
            ctx->batch_host = nullptr;
            ctx->batch_host_bytes = 0;
            void* h = nullptr;
            if (cudaMallocHost(&h, plan_bytes) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
            ctx->batch_host = (uint8_t*)h;
            ctx->batch_host_bytes = plan_bytes;
        }
        uint8_t* hp = ctx->batch_host;
        memcpy(hp + o_args, args.data(), sizeof(CompressArgs) * kb);
        memcpy(hp + o_tiles, tiles.data(), sizeof(uint32_t) * (ks + 1));
        memcpy(hp + o_groups, qgroups.data(), sizeof(uint32_t) * (ks + 1));
        memcpy(hp + o_off, off.data(), sizeof(uint32_t) * off.size());
        // arm the per-array range accumulators of a new layout
        if (ctx->batch_layout_bytes != bytes || ctx->batch_k != kb || !ctx->batch_states_armed) {
            std::vector<ArrayState> init(kb);
            memset(init.data(), 0, sizeof(ArrayState) * kb);
            for (auto& a : init) { a.acc_min = 0xffffffffu; a.min_key = 0xffffffffu; }
            if (cudaMemcpy(base + o_state, init.data(), sizeof(ArrayState) * kb, cudaMemcpyHostToDevice) != cudaSuccess) {
                cudaGetLastError();
                return SZ_ERR_CUDA;
            }
            ctx->batch_states_armed = 1;
            ctx->batch_layout_bytes = bytes;
            ctx->batch_k = kb;
        }
        BatchPlan plan;
        plan.args = (const CompressArgs*)(base + o_args);
        plan.cnt = (BatchCounters*)(base + o_cnt);
        plan.range_tiles = (const uint32_t*)(base + o_tiles);
        plan.quant_groups = (const uint32_t*)(base + o_groups);
        plan.item_off = (const uint32_t*)(base + o_off);
        plan.k = ks;
        plan.next = (uint32_t*)(base + o_cnt + sizeof(BatchCounters) * ks);
        plan.err = ctx->d_err;
        // graph: plan copy and counter reset, then the persistent kernel (small
        // arrays) beside the per-phase launches (large arrays)
        if (ctx->bg_exec) cudaGraphExecDestroy(ctx->bg_exec);
        if (ctx->bg_graph) cudaGraphDestroy(ctx->bg_graph);
        ctx->bg_exec = nullptr;
        ctx->bg_graph = nullptr;
        ctx->bg_key = 0;
        cudaGraph_t g = nullptr;
        cudaGraphNode_t n_copy, n_reset, n_kern;
        void* func;
        unsigned grid, block;
        size_t smem;
        batch_compress_config(&func, &grid, &block, &smem);
        cudaMemsetParams ms;
        memset(&ms, 0, sizeof(ms));
        ms.dst = base + o_cnt;
        ms.value = 0;
        ms.elementSize = 4;
        ms.width = cnt_bytes / 4;
        ms.height = 1;
        cudaKernelNodeParams kp{};
        void* kargs[] = {&plan};
        kp.func = func;
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = kargs;
        cudaGraphNode_t deps[2];
        if (cudaGraphCreate(&g, 0) != cudaSuccess ||
            cudaGraphAddMemcpyNode1D(&n_copy, g, nullptr, 0, base, hp, plan_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaGraphAddMemsetNode(&n_reset, g, nullptr, 0, &ms) != cudaSuccess) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            return SZ_ERR_CUDA;
        }
        deps[0] = n_copy;
        deps[1] = n_reset;
        KernelLaunch ml[8];
        const int nml = multi_compress_launches(plan.args, groups.data(), (int)groups.size(), ml, 8);
        bool nodes_ok = nml >= 0;
        cudaGraphNode_t prev = n_copy;
        for (int i = 0; nodes_ok && i < nml; ++i) {
            // range -> quantize -> codebook in a chain; the encoders after the codebook
            cudaKernelNodeParams mp{};
            void* margs[] = {&ml[i].args};
            mp.func = const_cast<void*>(ml[i].func);
            mp.gridDim = dim3(ml[i].grid[0], ml[i].grid[1], ml[i].grid[2]);
            mp.blockDim = dim3(ml[i].block[0], ml[i].block[1], ml[i].block[2]);
            mp.sharedMemBytes = (unsigned)ml[i].smem;
            mp.kernelParams = margs;
            cudaGraphNode_t node;
            nodes_ok = cudaGraphAddKernelNode(&node, g, &prev, 1, &mp) == cudaSuccess;
            if (i < 3) prev = node;
        }
        if (!nodes_ok || (ks && cudaGraphAddKernelNode(&n_kern, g, deps, 2, &kp) != cudaSuccess) ||
            cudaGraphInstantiate(&ctx->bg_exec, g, 0) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphDestroy(g);
            ctx->bg_exec = nullptr;
            return SZ_ERR_CUDA;
        }
        ctx->bg_graph = g;
        ctx->bg_key = key;
    }
    if (!ctx->prof_on) {
        if (cudaGraphLaunch(ctx->bg_exec, s) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    } else {
        // tracing: the graph's work as direct launches (same kernels, same
        // order) with an event pair around each, so each kernel is timed
        uint8_t* hp = ctx->batch_host;
        if (cudaMemcpyAsync(base, hp, plan_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(base + o_cnt, 0, cnt_bytes, s) != cudaSuccess) {
            cudaGetLastError();
            return SZ_ERR_CUDA;
        }
        if (ks) {
            BatchPlan plan;
            plan.args = (const CompressArgs*)(base + o_args);
            plan.cnt = (BatchCounters*)(base + o_cnt);
            plan.range_tiles = (const uint32_t*)(base + o_tiles);
            plan.quant_groups = (const uint32_t*)(base + o_groups);
            plan.item_off = (const uint32_t*)(base + o_off);
            plan.k = ks;
            plan.next = (uint32_t*)(base + o_cnt + sizeof(BatchCounters) * ks);
            plan.err = ctx->d_err;
            ProfScope pr(ctx, SZ_PHASE_BATCH, s);
            launch_batch_compress(plan, s);
        }
        KernelLaunch ml[8];
        const int nml = multi_compress_launches((const CompressArgs*)(base + o_args), groups.data(), (int)groups.size(),
                                                ml, 8);
        if (nml < 0) return SZ_ERR_ARG;
        for (int i = 0; i < nml; ++i) {
            ProfScope pr(ctx, ml[i].phase, s);
            void* margs[] = {&ml[i].args};
            if (cudaLaunchKernel(ml[i].func, dim3(ml[i].grid[0], ml[i].grid[1], ml[i].grid[2]),
                                 dim3(ml[i].block[0], ml[i].block[1], ml[i].block[2]), margs, ml[i].smem,
                                 s) != cudaSuccess) {
                cudaGetLastError();
                return SZ_ERR_CUDA;
            }
        }
    }
    if (cudaEventRecord(ctx->bg_done, s) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    if (out_bytes)
        for (uint32_t j = 0; j < kb; ++j)
            if ((st = queue_result(ctx, &args[j].st->total_bytes, &out_bytes[batched[j]], s)) != SZ_OK) return st;
    return SZ_OK;
}

sz_status batch_decompress(sz_ctx* ctx, int k, const void* const* d_in, const size_t* in_bytes, float* const* d_out,
                           const size_t* n_cap, size_t* n_out, cudaStream_t s) {
    cudaSetDevice(ctx->device);
    for (int i = 0; i < k; ++i)
        if (!d_in[i] || ((uintptr_t)d_in[i] & 15u) || (n_cap[i] && !d_out[i]) || ((uintptr_t)d_out[i] & 3u))
            return SZ_ERR_ARG;
    if (k == 0) return SZ_OK;
    if (k == 1) {
        DecompressArgs d = make_decompress_args(ctx, 0, d_in[0], in_bytes[0], d_out[0], n_cap[0]);
        return enqueue_decompress(ctx, d, n_out ? &n_out[0] : nullptr, s);
    }
    // ---- pool: args | units | unit offsets | per-stream state, tables, scratch ----------
    size_t bytes = 0;
    auto take = [&](size_t b) { size_t o = bytes; bytes += align256(b); return o; };
    const size_t o_args = take(sizeof(DecompressArgs) * k);
    const size_t plan_bytes = bytes;
    const size_t o_units = take(sizeof(uint32_t) * 2 * k);
    const size_t o_uoff = take(sizeof(uint64_t) * (k + 1));
    const size_t o_state = take(sizeof(ArrayState) * k);
    const size_t per = align256(sizeof(uint32_t) * kLutWords) + align256(sizeof(uint16_t) * 65536) +
                       align256(sizeof(uint32_t) * 4 * 65536);
    const size_t o_tab = take(per * k);
    if (bytes > ctx->dbatch_bytes) {
        if (cudaStreamSynchronize(s) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return SZ_ERR_CUDA;
        if (ctx->dbatch_pool) cudaFree(ctx->dbatch_pool);
        ctx->dbatch_pool = nullptr;
        ctx->dbatch_bytes = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
        ctx->dbatch_pool = (uint8_t*)p;
        ctx->dbatch_bytes = bytes;
    }
    // the previous call's plan copy must be done before the staging is reused
    if (ctx->dbatch_done && cudaEventSynchronize(ctx->dbatch_done) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    if (!ctx->dbatch_done && cudaEventCreateWithFlags(&ctx->dbatch_done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    if (plan_bytes > ctx->dbatch_host_bytes) {
        if (ctx->dbatch_host) cudaFreeHost(ctx->dbatch_host);
        ctx->dbatch_host = nullptr;
        ctx->dbatch_host_bytes = 0;
        void* h = nullptr;
        if (cudaMallocHost(&h, plan_bytes) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_NOMEM; }
        ctx->dbatch_host = (uint8_t*)h;
        ctx->dbatch_host_bytes = plan_bytes;
    }
    uint8_t* base = ctx->dbatch_pool;
    DecompressArgs* h_args = reinterpret_cast<DecompressArgs*>(ctx->dbatch_host + o_args);
    for (int i = 0; i < k; ++i) {
        DecompressArgs& d = h_args[i];
        memset(&d, 0, sizeof(d));
        uint8_t* t = base + o_tab + per * (size_t)i;
        d.in = (const uint8_t*)d_in[i];
        d.in_bytes = in_bytes[i];
        d.out = d_out[i];
        d.n_cap = n_cap[i];
        d.st = reinterpret_cast<ArrayState*>(base + o_state) + i;
        d.lut = reinterpret_cast<uint32_t*>(t);
        d.by_len = reinterpret_cast<uint16_t*>(t + align256(sizeof(uint32_t) * kLutWords));
        d.cb_scratch = reinterpret_cast<uint32_t*>(t + align256(sizeof(uint32_t) * kLutWords) +
                                                   align256(sizeof(uint16_t) * 65536));
        d.err = ctx->d_err;
    }
    if (cudaMemcpyAsync(base + o_args, h_args, sizeof(DecompressArgs) * k, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(ctx->dbatch_done, s) != cudaSuccess) {
        cudaGetLastError();
        return SZ_ERR_CUDA;
    }
    const DecompressArgs* d_args = reinterpret_cast<const DecompressArgs*>(base + o_args);
    uint64_t* d_uoff = reinterpret_cast<uint64_t*>(base + o_uoff);
    {
        ProfScope pr(ctx, SZ_PHASE_DECODE_SETUP, s);
        launch_decode_multi_setup(d_args, (uint32_t)k, reinterpret_cast<uint32_t*>(base + o_units), d_uoff, s);
    }
    {
        ProfScope pr(ctx, SZ_PHASE_DECODE, s);
        launch_decode_multi(d_args, (uint32_t)k, reinterpret_cast<uint32_t*>(base + o_units), d_uoff, s);
    }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    if (n_out)
        for (int i = 0; i < k; ++i) {
            sz_status st = queue_result(ctx, &h_args[i].st->n_out, &n_out[i], s);
            if (st != SZ_OK) return st;
        }
    return SZ_OK;
}

}  // namespace szg
