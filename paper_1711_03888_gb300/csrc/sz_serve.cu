// sz_serve.cu -- the serving loop: continuous batching of compress and
// decompress requests on one GPU (the in-situ setting of Sec. I / Sec. III,
// where every rank compresses the data it holds in memory).
//
// One host thread per context runs the loop:
//   retire  -- slots whose completion callback fired are read back (result
//              size, error word) and freed, with their budget bytes;
//   admit   -- queued requests are taken in arrival order while a slot is free
//              and the request's bytes fit the budget; a service-owned output
//              is carved from the device arena; the request's kernels are
//              enqueued on the slot's stream, so requests overlap on the device.
// Each slot owns a stream and a private workspace context: a request runs
// exactly the kernels of the plain call, so its output is the same alone and
// in the mix.  With a budget, a compress request's size-dependent scratch
// (code buffer, chunk tables) is carved from the arena with its output and
// counted in its budget bytes, so the slots' workspaces keep the size they
// were created with and admitting a request never synchronizes the device.  Completion is signalled by a host callback on the slot's stream
// (it only bumps a counter and wakes the loop; it takes no lock, so a loop that
// holds the lock across a device synchronize cannot deadlock with it).
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>
#include "sz_ctx.h"

using namespace szg;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kArenaAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over one device block.  Free ranges are kept by offset
// and merged with their neighbours on release.
struct Arena {
    uint8_t* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_by_off;   // offset -> length
    std::unordered_map<uintptr_t, size_t> live;   // address -> length

    void init(uint8_t* b, size_t s) {
        base = b;
        size = s;
        free_by_off.clear();
        live.clear();
        if (s) free_by_off[0] = s;
    }
    void* alloc(size_t bytes) {
        bytes = align_up(bytes ? bytes : 1, kArenaAlign);
        for (auto it = free_by_off.begin(); it != free_by_off.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, len = it->second;
            free_by_off.erase(it);
            if (len > bytes) free_by_off[off + bytes] = len - bytes;
            live[(uintptr_t)(base + off)] = bytes;
            return base + off;
        }
        return nullptr;
    }
    // returns the bytes freed, 0 if p is not a live allocation
    size_t release(void* p) {
        auto lv = live.find((uintptr_t)p);
        if (lv == live.end()) return 0;
        const size_t bytes = lv->second;
        live.erase(lv);
        size_t off = (uint8_t*)p - base, len = bytes;
        auto nx = free_by_off.lower_bound(off);
        if (nx != free_by_off.end() && off + len == nx->first) {
            len += nx->second;
            nx = free_by_off.erase(nx);
        }
        if (nx != free_by_off.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                off = pv->first;
                len += pv->second;
                free_by_off.erase(pv);
            }
        }
        free_by_off[off] = len;
        return bytes;
    }
};

// Device scratch of one compress request: its u16 code buffer (whole chunks)
// and its per-chunk escape counts and look-back words.  With a budget these
// come from the arena, so a slot's own workspace never grows while serving.
struct ReqScratch {
    size_t codes, cesc, cst, total;
};
ReqScratch compress_scratch(size_t n) {
    uint32_t C = 4096, G = 64;
    resolve_params(nullptr, n, &C, &G);
    const size_t nc = (n + C - 1) / C;
    ReqScratch r;
    r.codes = 0;
    r.cesc = align_up(2 * nc * C + 16, kArenaAlign);
    r.cst = r.cesc + align_up(4 * (nc + 1), kArenaAlign);
    r.total = r.cst + align_up(8 * (nc + 1), kArenaAlign);
    return r;
}

// Budget bytes one request holds while it runs (input, output, scratch).
size_t request_bytes(const sz_request& r) {
    const size_t n = r.n;
    if (r.op == SZ_OP_COMPRESS) {
        const size_t out = r.out ? r.out_cap : sz_max_compressed_bytes(n);
        return 4 * n + align_up(out, kArenaAlign) + compress_scratch(n).total;
    }
    return r.in_bytes + align_up(4 * n, kArenaAlign);
}

// Bytes of the output that stay held after completion (service-owned only).
size_t held_after(const sz_request& r) {
    if (r.out) return 0;
    return align_up(r.op == SZ_OP_COMPRESS ? sz_max_compressed_bytes(r.n) : 4 * r.n, kArenaAlign);
}

struct Pending {
    uint64_t ticket;
    sz_request req;
    double t_submit;
    size_t bytes;
};

struct Slot {
    sz_ctx* ws = nullptr;          // private workspace context
    cudaStream_t stream = nullptr;
    bool busy = false;
    uint64_t ticket = 0;
    double t_submit = 0;
    size_t bytes = 0, keep = 0;
    void* out = nullptr;
    uint8_t* scratch = nullptr;    // arena block of a compress request's codes and chunk tables
    uint64_t* h_res = nullptr;     // pinned: result size, error word
    std::atomic<int> fired{0};     // set by the completion callback
    struct sz_serve_state* owner = nullptr;
};

sz_status err_status(uint32_t err) {
    if (err & E_TIMEOUT) return SZ_ERR_TIMEOUT;
    if (err & E_CORRUPT) return SZ_ERR_CORRUPT;
    if (err & E_UNSUPPORTED) return SZ_ERR_UNSUPPORTED;
    if (err & E_CAPACITY) return SZ_ERR_CAPACITY;
    if (err) return SZ_ERR_CUDA;
    return SZ_OK;
}

}  // namespace

struct sz_serve_state {
    sz_ctx* ctx = nullptr;
    std::vector<Slot> slots;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, sz_result> results;
    std::mutex mu;
    std::condition_variable wake;      // loop: submissions and completions
    std::condition_variable done_cv;   // waiters: results
    std::atomic<uint64_t> fired_seq{0};
    std::thread loop;
    bool stopping = false;
    uint64_t next_ticket = 1;
    uint64_t budget_wait_ticket = 0;
    size_t budget = 0, held = 0;
    int active = 0;
    Arena arena;
    void* arena_mem = nullptr;
    sz_serve_counters c{};
};

namespace {

void CUDART_CB on_done(void* p) {
    Slot* s = (Slot*)p;
    s->fired.store(1, std::memory_order_release);
    s->owner->fired_seq.fetch_add(1, std::memory_order_release);
    s->owner->wake.notify_one();
}

// enqueue one request on a slot: the plain call's kernels, then the result copies.
// share: the request's persistent launches take 1/share of the GPU, so that
// requests in flight together split it instead of queueing behind each other.
// scratch: the request's arena block (compress_scratch layout), or null
// without a budget -- then the slot's workspace grows to the request, which
// synchronizes the device when it does.
sz_status launch_request(Slot& s, const sz_request& r, void* out, uint8_t* scratch, uint32_t share) {
    sz_ctx* w = s.ws;
    cudaSetDevice(w->device);
    w->grid_div = share;
    sz_status st;
    if (r.op == SZ_OP_COMPRESS) {
        uint32_t C, G;
        if ((st = resolve_params(nullptr, r.n, &C, &G)) != SZ_OK) return st;
        if (!scratch &&
            (st = ctx_reserve(w, 1, (r.n + C - 1) / C, (uint64_t)((r.n + C - 1) / C) * C)) != SZ_OK)
            return st;
        const size_t cap = r.out ? r.out_cap : sz_max_compressed_bytes(r.n);
        CompressArgs a = make_compress_args(w, 0, (const float*)r.in, r.n, r.eb, (int)r.kind, C, G, 0u, out, cap);
        if (scratch) {
            const ReqScratch L = compress_scratch(r.n);
            a.codes = reinterpret_cast<uint16_t*>(scratch + L.codes);
            a.chunk_esc = reinterpret_cast<uint32_t*>(scratch + L.cesc);
            a.chunk_status = reinterpret_cast<unsigned long long*>(scratch + L.cst);
        }
        if (cudaMemsetAsync(w->d_err, 0, sizeof(uint32_t), s.stream) != cudaSuccess) return SZ_ERR_CUDA;
        launch_range(&a, 1, s.stream);
        launch_quant(&a, 1, s.stream);
        launch_codebook(&a, 1, s.stream);
        if (a.n) launch_encode(&a, 1, s.stream);
        cudaMemcpyAsync(&s.h_res[0], &a.st->total_bytes, 8, cudaMemcpyDeviceToHost, s.stream);
    } else {
        DecompressArgs d = make_decompress_args(w, 0, r.in, r.in_bytes, (float*)out, r.n);
        if (cudaMemsetAsync(w->d_err, 0, sizeof(uint32_t), s.stream) != cudaSuccess) return SZ_ERR_CUDA;
        launch_decode_setup(&d, 1, s.stream);
        launch_decode(&d, 1, s.stream);
        cudaMemcpyAsync(&s.h_res[0], &d.st->n_out, 8, cudaMemcpyDeviceToHost, s.stream);
    }
    cudaMemcpyAsync(&s.h_res[1], w->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s.stream);
    s.fired.store(0, std::memory_order_relaxed);
    if (cudaLaunchHostFunc(s.stream, on_done, &s) != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    if (cudaPeekAtLastError() != cudaSuccess) { cudaGetLastError(); return SZ_ERR_CUDA; }
    return SZ_OK;
}

void finish(sz_serve_state* S, Slot& s, sz_status status, size_t out_size) {
    sz_result res;
    res.status = status;
    res.out_size = out_size;
    res.latency_s = now_s() - s.t_submit;
    res.out = s.out;
    if (status != SZ_OK && s.keep) {   // a failed request keeps no service buffer
        S->arena.release(s.out);
        res.out = nullptr;
        S->held -= s.keep;
    }
    S->results[s.ticket] = res;
    S->held -= s.bytes - s.keep;
    if (s.scratch) S->arena.release(s.scratch);
    s.scratch = nullptr;
    s.busy = false;
    s.out = nullptr;
    S->active--;
    S->c.completed++;
}

void serve_loop(sz_serve_state* S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    uint64_t seen = 0;
    for (;;) {
        bool retired = false, admitted = false;
        seen = S->fired_seq.load(std::memory_order_acquire);
        for (Slot& s : S->slots) {
            if (!s.busy || !s.fired.load(std::memory_order_acquire)) continue;
            // the callback runs after every earlier command of the stream
            cudaError_t q = cudaStreamQuery(s.stream);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            finish(S, s, q == cudaSuccess ? err_status((uint32_t)s.h_res[1]) : SZ_ERR_CUDA, (size_t)s.h_res[0]);
            retired = true;
        }
        if (retired) S->done_cv.notify_all();
        while (!S->queue.empty()) {
            Pending& p = S->queue.front();
            Slot* free_slot = nullptr;
            for (Slot& s : S->slots)
                if (!s.busy) { free_slot = &s; break; }
            if (!free_slot) break;
            if (S->budget && S->held + p.bytes > S->budget) {
                // wait for completions (or, with nothing in flight, the caller's releases)
                if (p.ticket != S->budget_wait_ticket) {
                    S->budget_wait_ticket = p.ticket;
                    S->c.budget_waits++;
                }
                break;
            }
            void* out = p.req.out;
            const size_t keep = held_after(p.req);
            if (!out) {
                out = S->arena.alloc(keep);
                if (!out) break;   // fragmented: wait for a release or a completion
            }
            uint8_t* scratch = nullptr;
            if (S->budget && p.req.op == SZ_OP_COMPRESS) {
                scratch = (uint8_t*)S->arena.alloc(compress_scratch(p.req.n).total);
                if (!scratch) {
                    if (!p.req.out) S->arena.release(out);
                    break;
                }
            }
            Slot& s = *free_slot;
            s.busy = true;
            s.ticket = p.ticket;
            s.t_submit = p.t_submit;
            s.bytes = p.bytes;
            s.keep = keep;
            s.out = out;
            s.scratch = scratch;
            S->held += p.bytes;
            S->active++;
            const sz_request r = p.req;
            S->queue.pop_front();
            if ((uint32_t)S->active > S->c.peak_inflight) S->c.peak_inflight = (uint32_t)S->active;
            if (S->held > S->c.peak_bytes) S->c.peak_bytes = S->held;
            const sz_status st = launch_request(s, r, out, scratch, (uint32_t)(S->active < 8 ? S->active : 8));
            if (st != SZ_OK) finish(S, s, st, 0);
            admitted = true;
        }
        if (S->stopping && S->active == 0 && !admitted) {
            // stopping with nothing in flight: what is still queued waits for
            // budget that only the caller's releases could free -- cancel it
            for (const Pending& p : S->queue) {
                sz_result res;
                res.status = SZ_ERR_BUSY;
                res.out_size = 0;
                res.latency_s = now_s() - p.t_submit;
                res.out = nullptr;
                S->results[p.ticket] = res;
            }
            S->queue.clear();
            break;
        }
        if (!retired && !admitted) {
            S->wake.wait_for(lk, std::chrono::microseconds(S->active ? 200 : 5000), [&] {
                return S->fired_seq.load(std::memory_order_acquire) != seen || S->stopping;
            });
        }
    }
    S->done_cv.notify_all();
}

sz_status take_result(sz_serve_state* S, uint64_t ticket, sz_result* res) {
    auto it = S->results.find(ticket);
    if (it == S->results.end()) {
        if (ticket == 0 || ticket >= S->next_ticket) return SZ_ERR_ARG;
        res->status = SZ_ERR_BUSY;
        res->out_size = 0;
        res->latency_s = 0;
        res->out = nullptr;
        return SZ_OK;
    }
    *res = it->second;
    S->results.erase(it);
    return SZ_OK;
}

}  // namespace

extern "C" {

sz_status sz_serve_start(sz_ctx* ctx, int slots) {
    if (!ctx || slots < 1 || slots > 64) return SZ_ERR_ARG;
    if (ctx->serve) return SZ_ERR_ARG;
    cudaSetDevice(ctx->device);
    sz_serve_state* S = new sz_serve_state();
    S->ctx = ctx;
    S->budget = ctx->budget;
    S->slots = std::vector<Slot>(slots);
    sz_status st = SZ_OK;
    if (S->budget) {
        if (cudaMalloc(&S->arena_mem, S->budget) != cudaSuccess) {
            cudaGetLastError();
            S->arena_mem = nullptr;
            st = SZ_ERR_NOMEM;
        } else {
            S->arena.init((uint8_t*)S->arena_mem, S->budget);
        }
    }
    for (Slot& s : S->slots) {
        if (st != SZ_OK) break;
        s.owner = S;
        if ((st = sz_ctx_create(&s.ws, ctx->device, 0)) != SZ_OK) break;
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&s.h_res, 2 * sizeof(uint64_t)) != cudaSuccess) {
            cudaGetLastError();
            st = SZ_ERR_CUDA;
        }
    }
    if (st != SZ_OK) {
        for (Slot& t : S->slots) {
            if (t.ws) sz_ctx_destroy(t.ws);
            if (t.stream) cudaStreamDestroy(t.stream);
            if (t.h_res) cudaFreeHost(t.h_res);
        }
        if (S->arena_mem) cudaFree(S->arena_mem);
        delete S;
        return st;
    }
    ctx->serve = S;
    S->loop = std::thread(serve_loop, S);
    return SZ_OK;
}

sz_status sz_serve_submit(sz_ctx* ctx, const sz_request* req, uint64_t* ticket) {
    if (!ctx || !ctx->serve || !req || !ticket) return SZ_ERR_ARG;
    const sz_request& r = *req;
    sz_serve_state* S = ctx->serve;
    if (r.op == SZ_OP_COMPRESS) {
        // the plain call's checks; a service-owned output is 256-byte aligned
        void* out_check = r.out ? r.out : (void*)(uintptr_t)kArenaAlign;
        if (validate_compress((const float*)r.in, r.n, r.eb, r.kind, out_check) != SZ_OK) return SZ_ERR_ARG;
        uint32_t C, G;
        if (resolve_params(nullptr, r.n, &C, &G) != SZ_OK) return SZ_ERR_ARG;
    } else if (r.op == SZ_OP_DECOMPRESS) {
        if (!r.in || ((uintptr_t)r.in & 15u) || (r.out && ((uintptr_t)r.out & 3u))) return SZ_ERR_ARG;
    } else {
        return SZ_ERR_ARG;
    }
    if (!r.out && !S->budget) return SZ_ERR_ARG;   // no arena to take the output from
    const size_t bytes = request_bytes(r);
    if (S->budget && bytes > S->budget) return SZ_ERR_BUSY;   // could never be admitted
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) return SZ_ERR_ARG;
        Pending p;
        p.ticket = S->next_ticket++;
        p.req = r;
        p.t_submit = now_s();
        p.bytes = bytes;
        S->queue.push_back(p);
        S->c.submitted++;
        if ((uint32_t)S->queue.size() > S->c.peak_queue) S->c.peak_queue = (uint32_t)S->queue.size();
        *ticket = p.ticket;
    }
    S->fired_seq.fetch_add(1, std::memory_order_release);
    S->wake.notify_one();
    return SZ_OK;
}

sz_status sz_serve_poll(sz_ctx* ctx, uint64_t ticket, sz_result* res) {
    if (!ctx || !ctx->serve || !res) return SZ_ERR_ARG;
    sz_serve_state* S = ctx->serve;
    std::lock_guard<std::mutex> lk(S->mu);
    return take_result(S, ticket, res);
}

sz_status sz_serve_wait(sz_ctx* ctx, uint64_t ticket, double timeout_s, sz_result* res) {
    if (!ctx || !ctx->serve || !res || !(timeout_s >= 0.0)) return SZ_ERR_ARG;
    sz_serve_state* S = ctx->serve;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket == 0 || ticket >= S->next_ticket) return SZ_ERR_ARG;
    const auto limit = std::chrono::steady_clock::now() +
                       std::chrono::microseconds((long long)(timeout_s > 1e6 ? 1e12 : timeout_s * 1e6));
    S->done_cv.wait_until(lk, limit, [&] { return S->results.count(ticket) != 0; });
    return take_result(S, ticket, res);
}

sz_status sz_serve_release(sz_ctx* ctx, void* out) {
    if (!ctx || !ctx->serve || !out) return SZ_ERR_ARG;
    sz_serve_state* S = ctx->serve;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const size_t b = S->arena.release(out);
        if (!b) return SZ_ERR_ARG;
        S->held -= b;
    }
    S->fired_seq.fetch_add(1, std::memory_order_release);
    S->wake.notify_one();
    return SZ_OK;
}

sz_status sz_serve_stats(sz_ctx* ctx, sz_serve_counters* out) {
    if (!ctx || !ctx->serve || !out) return SZ_ERR_ARG;
    std::lock_guard<std::mutex> lk(ctx->serve->mu);
    *out = ctx->serve->c;
    return SZ_OK;
}

sz_status sz_serve_stop(sz_ctx* ctx) {
    if (!ctx) return SZ_ERR_ARG;
    sz_serve_state* S = ctx->serve;
    if (!S) return SZ_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->fired_seq.fetch_add(1, std::memory_order_release);
    S->wake.notify_one();
    if (S->loop.joinable()) S->loop.join();
    cudaSetDevice(ctx->device);
    for (Slot& s : S->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.ws) sz_ctx_destroy(s.ws);
        if (s.stream) cudaStreamDestroy(s.stream);
        if (s.h_res) cudaFreeHost(s.h_res);
    }
    if (S->arena_mem) cudaFree(S->arena_mem);
    ctx->serve = nullptr;
    delete S;
    return SZ_OK;
}

}  // extern "C"
