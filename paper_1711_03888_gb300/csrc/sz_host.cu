// sz_host.cu -- compression and decompression of arrays held in host memory.
//
// The paper's in-situ setting (Sec. I, Sec. III) hands the compressor arrays
// that live in the simulation's memory; on a Grace-Blackwell node that can be
// the CPU side of the NVLink-C2C link.  These two calls take host arrays and
// produce host arrays, and keep the link busy: the arrays are cut into groups
// of at least kGroupBytes input bytes, and the groups flow through two device
// staging slots on three streams,
//
//     copy-in stream   host -> slot s            (group g)
//     compute stream   compress / decompress     (group g - 1, the other slot)
//     copy-out stream  slot s' -> host           (group g - 2 ... )
//
// so the host->device copy of one group, the kernels of the previous one and
// the device->host copy of the one before overlap.  Every array goes through
// the per-array path (the same kernels and the same bytes as sz_compress /
// sz_decompress) on the context's workspace slot 0, in stream order.
//
// Compression learns a stream's size on the device, so the host waits for
// each group's kernels (one event) before it queues that group's copy-out;
// the next group's copy-in and kernels are already queued by then.
// Decompression reads each stream's element count from its header in host
// memory and never waits.  Both calls end with sz_sync() on the compute
// stream and return its status.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <vector>
#include "../../include/sz_gb300.h"
#include "sz_internal.h"
#include "sz_ctx.h"

using namespace szg;

namespace {

constexpr size_t kGroupBytes = 64ull << 20;    // a group closes once it holds this many input bytes
constexpr int kSlots = 2;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

sz_status cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return SZ_OK;
    cudaGetLastError();
    return SZ_ERR_CUDA;
}

// streams, events and the pinned result array, created on first use
sz_status host_setup(sz_ctx* ctx, int k) {
    if (!ctx->host_h2d && cuda_ok(cudaStreamCreateWithFlags(&ctx->host_h2d, cudaStreamNonBlocking)) != SZ_OK)
        return SZ_ERR_CUDA;
    if (!ctx->host_d2h && cuda_ok(cudaStreamCreateWithFlags(&ctx->host_d2h, cudaStreamNonBlocking)) != SZ_OK)
        return SZ_ERR_CUDA;
    for (int s = 0; s < kSlots; ++s)
        for (int j = 0; j < 3; ++j)
            if (!ctx->host_ev[s][j] &&
                cuda_ok(cudaEventCreateWithFlags(&ctx->host_ev[s][j], cudaEventDisableTiming)) != SZ_OK)
                return SZ_ERR_CUDA;
    if ((size_t)k > ctx->host_pin_cap) {
        if (ctx->host_pin) cudaFreeHost(ctx->host_pin);
        ctx->host_pin = nullptr;
        ctx->host_pin_cap = 0;
        const size_t cap = (size_t)k < 1024 ? 1024 : (size_t)k;
        if (cudaMallocHost(&ctx->host_pin, sizeof(uint64_t) * cap) != cudaSuccess) {
            cudaGetLastError();
            return SZ_ERR_NOMEM;
        }
        ctx->host_pin_cap = cap;
    }
    return SZ_OK;
}

// device staging: kSlots x (input region + output region)
sz_status host_pool(sz_ctx* ctx, size_t in_bytes, size_t out_bytes, uint8_t** in, uint8_t** out) {
    const size_t slot = align256(in_bytes) + align256(out_bytes);
    const size_t need = kSlots * slot;
    if (need > ctx->host_pool_bytes) {
        // the previous host call has finished with the old pool (both calls are synchronous)
        if (ctx->host_pool) cudaFree(ctx->host_pool);
        ctx->host_pool = nullptr;
        ctx->host_pool_bytes = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return SZ_ERR_NOMEM;
        }
        ctx->host_pool = (uint8_t*)p;
        ctx->host_pool_bytes = need;
    }
    for (int s = 0; s < kSlots; ++s) {
        in[s] = ctx->host_pool + s * slot;
        out[s] = in[s] + align256(in_bytes);
    }
    return SZ_OK;
}

// consecutive arrays, each group closing at kGroupBytes of input
struct Group {
    int first, last;        // arrays [first, last)
};

std::vector<Group> make_groups(int k, const std::vector<size_t>& in_bytes) {
    std::vector<Group> g;
    size_t acc = 0;
    for (int i = 0; i < k; ++i) {
        if (g.empty() || acc >= kGroupBytes) {
            g.push_back(Group{i, i});
            acc = 0;
        }
        g.back().last = i + 1;
        acc += in_bytes[i];
    }
    return g;
}

// per-slot byte offsets of each array's input and output within its group
void slot_offsets(const std::vector<Group>& groups, const std::vector<size_t>& a_bytes,
                  const std::vector<size_t>& b_bytes, std::vector<size_t>& a_off, std::vector<size_t>& b_off,
                  size_t* a_max, size_t* b_max) {
    *a_max = *b_max = 0;
    for (const Group& g : groups) {
        size_t a = 0, b = 0;
        for (int i = g.first; i < g.last; ++i) {
            a_off[i] = a;
            b_off[i] = b;
            a += align256(a_bytes[i]);
            b += align256(b_bytes[i]);
        }
        if (a > *a_max) *a_max = a;
        if (b > *b_max) *b_max = b;
    }
}

// element count of a stream from its header (0 when it is not a version-1 stream)
uint64_t header_elems(const void* h, size_t bytes) {
    if (!h || bytes < kHeaderBytes) return 0;
    const uint8_t* p = (const uint8_t*)h;
    uint32_t magic;
    uint16_t version;
    uint64_t n;
    memcpy(&magic, p + H_MAGIC, 4);
    memcpy(&version, p + H_VERSION, 2);
    memcpy(&n, p + H_N, 8);
    return (magic == kMagic && version == kVersion) ? n : 0;
}

// waits for the copy streams, then sz_sync on the compute stream
sz_status host_finish(sz_ctx* ctx, cudaStream_t cs, sz_status st) {
    const cudaError_t e1 = cudaStreamSynchronize(ctx->host_h2d);
    const cudaError_t e2 = cudaStreamSynchronize(ctx->host_d2h);
    const sz_status s3 = sz_sync(ctx, cs);
    if (st != SZ_OK) return st;
    if (e1 != cudaSuccess || e2 != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return s3;
}

}  // namespace

void sz_ctx::free_host() {
    if (cpc) cudaFree(cpc);
    cpc = nullptr;
    cpc_bytes = 0;
    if (host_pool) cudaFree(host_pool);
    host_pool = nullptr;
    host_pool_bytes = 0;
    if (host_pin) cudaFreeHost(host_pin);
    host_pin = nullptr;
    host_pin_cap = 0;
    for (auto& row : host_ev)
        for (cudaEvent_t& e : row) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    if (host_h2d) cudaStreamDestroy(host_h2d);
    if (host_d2h) cudaStreamDestroy(host_d2h);
    host_h2d = host_d2h = nullptr;
}

extern "C" {

sz_status sz_compress_host(sz_ctx* ctx, int k, const float* const* h_in, const size_t* n, const double* eb,
                           sz_eb_kind kind, const sz_params* params, void* const* h_out, const size_t* out_cap,
                           size_t* out_bytes, void* stream) {
    if (!ctx || k < 0 || (k && (!h_in || !n || !eb || !h_out || !out_cap || !out_bytes))) return SZ_ERR_ARG;
    if (k == 0) return SZ_OK;
    std::vector<uint32_t> Cs(k), Gs(k);
    std::vector<size_t> ib(k), ob(k);
    uint64_t max_chunks = 0, max_codes = 0;
    for (int i = 0; i < k; ++i) {
        if ((n[i] && !h_in[i]) || !h_out[i] || (uint64_t)n[i] >= (1ull << 32)) return SZ_ERR_ARG;
        if (!(eb[i] >= 0.0) || eb[i] > 1.7976931348623157e308 || (kind != SZ_EB_ABS && kind != SZ_EB_REL))
            return SZ_ERR_ARG;
        sz_status st = resolve_params(params, n[i], &Cs[i], &Gs[i]);
        if (st != SZ_OK) return st;
        ib[i] = 4 * n[i];
        ob[i] = sz_max_compressed_bytes(n[i]);
        const uint64_t nc = (n[i] + Cs[i] - 1) / Cs[i];
        if (nc > max_chunks) max_chunks = nc;
        if (nc * Cs[i] > max_codes) max_codes = nc * Cs[i];
    }
    cudaSetDevice(ctx->device);
    cudaStream_t cs = (cudaStream_t)stream;
    sz_status st = ctx_reserve(ctx, 1, max_chunks, max_codes);
    if (st != SZ_OK) return st;
    if ((st = host_setup(ctx, k)) != SZ_OK) return st;
    const std::vector<Group> groups = make_groups(k, ib);
    std::vector<size_t> ioff(k), ooff(k);
    size_t imax, omax;
    slot_offsets(groups, ib, ob, ioff, ooff, &imax, &omax);
    uint8_t* din[kSlots];
    uint8_t* dout[kSlots];
    if ((st = host_pool(ctx, imax, omax, din, dout)) != SZ_OK) return st;
    uint64_t* sizes = ctx->host_pin;
    cudaStream_t h2d = ctx->host_h2d, d2h = ctx->host_d2h;
    bool too_small = false;

    // copy-out of group g once its kernels are done (host wait on one event)
    auto drain = [&](size_t g) -> sz_status {
        const int s = (int)(g % kSlots);
        if (cudaEventSynchronize(ctx->host_ev[s][1]) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
        for (int i = groups[g].first; i < groups[g].last; ++i) {
            const size_t b = (size_t)sizes[i];
            out_bytes[i] = b;
            if (b > ob[i]) continue;                  // no stream (a device error, reported by sz_sync)
            if (b > out_cap[i]) { too_small = true; continue; }
            if (cuda_ok(cudaMemcpyAsync(h_out[i], dout[s] + ooff[i], b, cudaMemcpyDeviceToHost, d2h)) != SZ_OK)
                return SZ_ERR_CUDA;
        }
        return cuda_ok(cudaEventRecord(ctx->host_ev[s][2], d2h));
    };

    for (size_t g = 0; g < groups.size() && st == SZ_OK; ++g) {
        const int s = (int)(g % kSlots);
        cudaEvent_t ev_in = ctx->host_ev[s][0], ev_done = ctx->host_ev[s][1], ev_out = ctx->host_ev[s][2];
        // copy-in, once the kernels of group g - kSlots have finished reading this slot
        if (g >= kSlots && (st = cuda_ok(cudaStreamWaitEvent(h2d, ev_done, 0))) != SZ_OK) break;
        for (int i = groups[g].first; i < groups[g].last && st == SZ_OK; ++i)
            if (ib[i]) st = cuda_ok(cudaMemcpyAsync(din[s] + ioff[i], h_in[i], ib[i], cudaMemcpyHostToDevice, h2d));
        if (st != SZ_OK || (st = cuda_ok(cudaEventRecord(ev_in, h2d))) != SZ_OK) break;
        // kernels, once the copy-in is done and group g - kSlots has left the output region
        if ((st = cuda_ok(cudaStreamWaitEvent(cs, ev_in, 0))) != SZ_OK) break;
        if (g >= kSlots && (st = cuda_ok(cudaStreamWaitEvent(cs, ev_out, 0))) != SZ_OK) break;
        for (int i = groups[g].first; i < groups[g].last && st == SZ_OK; ++i) {
            CompressArgs a = make_compress_args(ctx, 0, (const float*)(din[s] + ioff[i]), n[i], eb[i], (int)kind,
                                                Cs[i], Gs[i], 0u, dout[s] + ooff[i], ob[i]);
            a.pred = params_pred(params);
            if ((st = enqueue_compress(ctx, a, nullptr, cs)) != SZ_OK) break;
            st = cuda_ok(cudaMemcpyAsync(&sizes[i], &a.st->total_bytes, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs));
        }
        if (st != SZ_OK || (st = cuda_ok(cudaEventRecord(ev_done, cs))) != SZ_OK) break;
        if (g >= 1) st = drain(g - 1);
    }
    if (st == SZ_OK) st = drain(groups.size() - 1);
    st = host_finish(ctx, cs, st);
    if (st == SZ_OK && too_small) st = SZ_ERR_CAPACITY;
    return st;
}

sz_status sz_decompress_host(sz_ctx* ctx, int k, const void* const* h_in, const size_t* in_bytes,
                             float* const* h_out, const size_t* n_cap, size_t* n_out, void* stream) {
    if (!ctx || k < 0 || (k && (!h_in || !in_bytes || !h_out || !n_cap || !n_out))) return SZ_ERR_ARG;
    if (k == 0) return SZ_OK;
    std::vector<size_t> ib(k), yb(k), ncopy(k);
    for (int i = 0; i < k; ++i) {
        if (!h_in[i] || (n_cap[i] && !h_out[i])) return SZ_ERR_ARG;
        const uint64_t nh = header_elems(h_in[i], in_bytes[i]);
        // a stream larger than the caller's buffer decodes into nothing and reports SZ_ERR_CAPACITY
        ncopy[i] = nh <= n_cap[i] ? (size_t)nh : 0;
        ib[i] = in_bytes[i];
        yb[i] = 4 * ncopy[i];
    }
    cudaSetDevice(ctx->device);
    cudaStream_t cs = (cudaStream_t)stream;
    sz_status st = host_setup(ctx, k);
    if (st != SZ_OK) return st;
    const std::vector<Group> groups = make_groups(k, ib);
    std::vector<size_t> ioff(k), yoff(k);
    size_t imax, ymax;
    slot_offsets(groups, ib, yb, ioff, yoff, &imax, &ymax);
    uint8_t* din[kSlots];
    uint8_t* dy[kSlots];
    if ((st = host_pool(ctx, imax, ymax, din, dy)) != SZ_OK) return st;
    uint64_t* counts = ctx->host_pin;
    for (int i = 0; i < k; ++i) counts[i] = 0;
    cudaStream_t h2d = ctx->host_h2d, d2h = ctx->host_d2h;

    for (size_t g = 0; g < groups.size() && st == SZ_OK; ++g) {
        const int s = (int)(g % kSlots);
        cudaEvent_t ev_in = ctx->host_ev[s][0], ev_done = ctx->host_ev[s][1], ev_out = ctx->host_ev[s][2];
        if (g >= kSlots && (st = cuda_ok(cudaStreamWaitEvent(h2d, ev_done, 0))) != SZ_OK) break;
        for (int i = groups[g].first; i < groups[g].last && st == SZ_OK; ++i)
            if (ib[i]) st = cuda_ok(cudaMemcpyAsync(din[s] + ioff[i], h_in[i], ib[i], cudaMemcpyHostToDevice, h2d));
        if (st != SZ_OK || (st = cuda_ok(cudaEventRecord(ev_in, h2d))) != SZ_OK) break;
        if ((st = cuda_ok(cudaStreamWaitEvent(cs, ev_in, 0))) != SZ_OK) break;
        if (g >= kSlots && (st = cuda_ok(cudaStreamWaitEvent(cs, ev_out, 0))) != SZ_OK) break;
        for (int i = groups[g].first; i < groups[g].last && st == SZ_OK; ++i) {
            DecompressArgs d = make_decompress_args(ctx, 0, din[s] + ioff[i], ib[i], (float*)(dy[s] + yoff[i]),
                                                    ncopy[i]);
            if ((st = enqueue_decompress(ctx, d, nullptr, cs)) != SZ_OK) break;
            st = cuda_ok(cudaMemcpyAsync(&counts[i], &d.st->n_out, sizeof(uint64_t), cudaMemcpyDeviceToHost, cs));
        }
        if (st != SZ_OK || (st = cuda_ok(cudaEventRecord(ev_done, cs))) != SZ_OK) break;
        // copy-out follows the kernels on the device; the host does not wait
        if ((st = cuda_ok(cudaStreamWaitEvent(d2h, ev_done, 0))) != SZ_OK) break;
        for (int i = groups[g].first; i < groups[g].last && st == SZ_OK; ++i)
            if (yb[i])
                st = cuda_ok(cudaMemcpyAsync(h_out[i], dy[s] + yoff[i], yb[i], cudaMemcpyDeviceToHost, d2h));
        if (st == SZ_OK) st = cuda_ok(cudaEventRecord(ev_out, d2h));
    }
    st = host_finish(ctx, cs, st);
    for (int i = 0; i < k; ++i) n_out[i] = (size_t)counts[i];
    return st;
}

}  // extern "C"
