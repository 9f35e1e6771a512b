// Serving runtime: continuous batching of bake and render requests over
// several resident scenes on one GPU.
//
//  * Admission.  The server owns one device arena of `hbm_budget` bytes.  A
//    request is admitted (in arrival order) when its device buffers fit in
//    the arena; one larger than the whole budget completes at once with
//    FIPT_ERR_BUDGET.  Inputs are copied in on a copy stream.
//  * Continuous batching.  Each batch takes chunks of up to `chunk_points`
//    points from the admitted bake requests (any scene) until
//    `max_batch_rays` rays -- the oldest request first, up to a quarter of
//    the batch, then the requests with the least remaining work -- and runs
//    them in one launch of the batched bake kernel; render requests run
//    their forward/backward kernels in the same batch.  Up to three batches
//    are in flight, so a request that arrives while others run joins the
//    next batch, and its work overlaps theirs on the device.  Chunks keep request-local Philox counters, so a result is
//    identical alone and in any mix.
//  * Completion.  When a request's last chunk has run, its outputs are
//    copied back on the copy stream and its arena space is freed.
//  * All waits are on the host (event queries with short sleeps, bounded by
//    the caller's timeouts); no kernel waits on anything.
//  * Failure.  A launch that fails, or a batch whose device work fails, stops
//    the server: no new work starts and every unfinished request ends with
//    that error once none of its copies or kernels is still queued.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fipt_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxChunks = 8192;   // descriptors per batch
constexpr int kSlots = 3;          // batches in flight

}  // namespace

// ---------------------------------------------------------------- arena (host bookkeeping)
// First-fit allocator over [0, size) with coalescing of free neighbours;
// 256-byte granularity.  Pure host logic; the server maps offsets onto its
// device buffer.
struct fipt_arena {
    size_t size, used = 0, peak = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    explicit fipt_arena(size_t s) : size(s & ~size_t(255)) {
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = up256(bytes ? bytes : 1);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t roff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[roff] = rest;
                used += bytes;
                peak = std::max(peak, used);
                return true;
            }
        }
        return false;
    }
    bool release(size_t off, size_t bytes) {
        bytes = up256(bytes ? bytes : 1);
        if (off + bytes > size) return false;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first < off + bytes) return false;          // overlaps a free block
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second > off) return false;
        }
        used -= bytes;
        size_t o = off, b = bytes;
        if (nx != free_.end() && nx->first == off + bytes) {
            b += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                o = pv->first;
                b += pv->second;
                free_.erase(pv);
            }
        }
        free_[o] = b;
        return true;
    }
    size_t largest_free() const {
        size_t m = 0;
        for (auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
};

extern "C" fipt_status fipt_arena_create(size_t bytes, fipt_arena** out) {
    FIPT_REQUIRE(out, "out is NULL");
    *out = new fipt_arena(bytes);
    return FIPT_OK;
}
extern "C" fipt_status fipt_arena_alloc(fipt_arena* a, size_t bytes, size_t* offset) {
    FIPT_REQUIRE(a && offset, "NULL argument");
    if (!a->alloc(bytes, offset)) return fipt_set_error(FIPT_ERR_BUDGET, "arena full");
    return FIPT_OK;
}
extern "C" fipt_status fipt_arena_free(fipt_arena* a, size_t offset, size_t bytes) {
    FIPT_REQUIRE(a, "NULL arena");
    FIPT_REQUIRE(a->release(offset, bytes), "free of a block that is not allocated");
    return FIPT_OK;
}
extern "C" fipt_status fipt_arena_info(fipt_arena* a, size_t* used, size_t* peak, size_t* largest) {
    FIPT_REQUIRE(a, "NULL arena");
    if (used) *used = a->used;
    if (peak) *peak = a->peak;
    if (largest) *largest = a->largest_free();
    return FIPT_OK;
}
extern "C" fipt_status fipt_arena_destroy(fipt_arena* a) {
    delete a;
    return FIPT_OK;
}

// ---------------------------------------------------------------- server
namespace {

enum State { PENDING, ADMITTED, LAUNCHED, COPYING, DONE };

struct Table {
    const float *Ld, *Ls0, *Ls1;
    int64_t N;
    int K;
    float grid[FIPT_MAX_K];
};

struct Req {
    uint64_t ticket = 0;
    fipt_request r{};
    State state = PENDING;
    fipt_status result = FIPT_OK;
    size_t off = 0, bytes = 0;
    char* base = nullptr;
    // device buffers inside the arena
    fipt_query* dq = nullptr;
    float *dLd = nullptr, *dLs0 = nullptr, *dLs1 = nullptr;
    float *da = nullptr, *dr = nullptr, *dm = nullptr, *dLgt = nullptr, *dLr = nullptr;
    float *dga = nullptr, *dgr = nullptr, *dgm = nullptr;
    double* dloss = nullptr;
    void* dws = nullptr;
    size_t ws_bytes = 0;
    int64_t next = 0;             // bake: next unscheduled point
    uint64_t last_batch = 0;      // batch that runs this request's last work
    cudaEvent_t h2d = nullptr, d2h = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Batch {
    uint64_t seq;
    int slot;
    cudaEvent_t done;
    std::vector<uint64_t> finishing;
};

}  // namespace

struct fipt_server {
    fipt_ctx* ctx = nullptr;
    size_t budget = 0;
    int64_t max_batch_rays = 0, chunk_points = 0;
    char* arena_dev = nullptr;
    fipt_arena* arena = nullptr;
    cudaStream_t compute = nullptr, copy = nullptr;
    int32_t* status = nullptr;                 // device status word of this server
    int32_t* status_host = nullptr;            // pinned, one per slot
    BakeChunk* chunk_dev[kSlots] = {};
    BakeChunk* chunk_host[kSlots] = {};        // pinned staging
    std::vector<fipt_scene*> scenes;
    std::vector<Table> tables;
    std::map<uint64_t, Req*> reqs;
    std::deque<uint64_t> pending;              // arrival order
    std::vector<uint64_t> active;              // admitted, work left to schedule (admission order)
    std::deque<Batch> inflight;
    std::vector<uint64_t> copying;
    uint64_t next_ticket = 1, next_batch = 1;
    // statistics
    uint64_t n_batches = 0, n_chunks = 0, max_reqs_in_batch = 0, rays = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    fipt_status fatal = FIPT_OK;
    uint64_t fatal_batch = 0;                  // first batch whose work is lost
    int64_t fail_after = -1;                   // test hook: batches left before a launch failure
    char fatal_msg[256] = "";

    void run();
    bool admit(Req* q);
    void launch_batch();
    void retire(Batch& b);
    void finish_copies();
    void drain_after_fatal();
    void set_fatal(fipt_status st, uint64_t batch, const char* msg);
};

namespace {

size_t request_bytes(const fipt_request& r, const fipt_server* s) {
    if (r.kind == FIPT_REQ_BAKE) {
        const size_t n = (size_t)r.n, K = (size_t)r.params.K;
        return up256(n * sizeof(fipt_query)) + up256(n * 3 * 4) + 2 * up256(n * K * 3 * 4) + 256;
    }
    size_t ws = 0;
    fipt_render_workspace_size(r.n, &ws);
    const size_t n = (size_t)r.n;
    (void)s;
    return 4 * up256(n * 12) + 4 * up256(n * 4) + up256(n * 12) + up256(8) + up256(ws) + 256;
}

}  // namespace

bool fipt_server::admit(Req* q) {
    size_t off;
    if (!arena->alloc(q->bytes, &off)) return false;
    q->off = off;
    q->base = arena_dev + off;
    Carver c{q->base, 0};
    const fipt_request& r = q->r;
    const size_t n = (size_t)r.n;
    if (r.kind == FIPT_REQ_BAKE) {
        const size_t K = (size_t)r.params.K;
        q->dq = c.take<fipt_query>(n);
        q->dLd = c.take<float>(n * 3);
        q->dLs0 = c.take<float>(n * K * 3);
        q->dLs1 = c.take<float>(n * K * 3);
        if (n) cudaMemcpyAsync(q->dq, r.queries, n * sizeof(fipt_query), cudaMemcpyHostToDevice, copy);
    } else {
        q->da = c.take<float>(n * 3);
        q->dr = c.take<float>(n);
        q->dm = c.take<float>(n);
        q->dLgt = c.take<float>(n * 3);
        q->dLr = c.take<float>(n * 3);
        q->dga = c.take<float>(n * 3);
        q->dgr = c.take<float>(n);
        q->dgm = c.take<float>(n);
        q->dloss = c.take<double>(1);
        fipt_render_workspace_size(r.n, &q->ws_bytes);
        q->dws = c.take<char>(q->ws_bytes);
        if (n) {
            cudaMemcpyAsync(q->da, r.albedo, n * 12, cudaMemcpyHostToDevice, copy);
            cudaMemcpyAsync(q->dr, r.rough, n * 4, cudaMemcpyHostToDevice, copy);
            cudaMemcpyAsync(q->dm, r.metal, n * 4, cudaMemcpyHostToDevice, copy);
            cudaMemcpyAsync(q->dLgt, r.Lgt, n * 12, cudaMemcpyHostToDevice, copy);
        }
    }
    cudaEventRecord(q->h2d, copy);
    q->state = ADMITTED;
    q->t_admit = now_s();
    return true;
}

void fipt_server::launch_batch() {
    const int slot = (int)(next_batch % kSlots);
    BakeChunk* H = chunk_host[slot];
    int nch = 0;
    int64_t warps = 0, batch_rays = 0;
    std::vector<uint64_t> involved, finishing;
    // render requests: all of their work runs in this batch
    for (uint64_t t : active) {
        Req* q = reqs[t];
        if (q->r.kind != FIPT_REQ_RENDER) continue;
        involved.push_back(t);
    }
    // bake requests: the oldest admitted request first takes up to a quarter
    // of the batch's rays (so no request starves), then the requests with the
    // least remaining work take chunks in that order (shortest remaining work
    // first keeps small requests' latency low), then the oldest again
    std::vector<uint64_t> order;
    for (uint64_t t : active) {
        Req* q = reqs[t];
        if (q->r.kind == FIPT_REQ_BAKE && q->next < q->r.n) order.push_back(t);
    }
    auto remaining = [&](uint64_t t) {
        const Req* q = reqs[t];
        const fipt_bake_params& P = q->r.params;
        return (q->r.n - q->next) * (P.spp_diffuse + (int64_t)P.K * P.spp_specular);
    };
    if (order.size() > 1)
        std::stable_sort(order.begin() + 1, order.end(),
                         [&](uint64_t a, uint64_t b) { return remaining(a) < remaining(b); });
    // takes chunks of request t while its share (rays) and the batch allow
    auto take = [&](uint64_t t, int64_t share) {
        Req* q = reqs[t];
        const fipt_bake_params& P = q->r.params;
        const int64_t rays_per_pt = P.spp_diffuse + (int64_t)P.K * P.spp_specular;
        int64_t got = 0;
        while (q->next < q->r.n && nch < kMaxChunks) {
            const int64_t c = std::min<int64_t>(chunk_points, q->r.n - q->next);
            if (nch > 0 && (batch_rays + c * rays_per_pt > max_batch_rays || got + c * rays_per_pt > share))
                break;
            BakeChunk& C = H[nch++];
            fipt_scene* sc = scenes[q->r.target];
            C.sc = sc->view();
            C.q = q->dq + q->next;
            C.Ld = q->dLd + 3 * q->next;
            C.Ls0 = q->dLs0 + q->next * P.K * 3;
            C.Ls1 = q->dLs1 + q->next * P.K * 3;
            C.n = c;
            C.warp_begin = warps;
            C.A.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
            C.A.request_id = P.request_id;
            C.A.point_base = (uint32_t)q->next;
            C.A.spp_d = P.spp_diffuse;
            C.A.spp_s = P.spp_specular;
            C.A.K = P.K;
            for (int k = 0; k < FIPT_MAX_K; ++k) C.A.sigma[k] = k < P.K ? P.sigma[k] : 1.0f;
            warps += ((c + 31) / 32) * (1 + P.K);
            batch_rays += c * rays_per_pt;
            got += c * rays_per_pt;
            q->next += c;
            if (std::find(involved.begin(), involved.end(), t) == involved.end()) involved.push_back(t);
        }
    };
    if (!order.empty()) {
        take(order[0], max_batch_rays / 4);
        for (size_t i = 1; i < order.size() && batch_rays < max_batch_rays && nch < kMaxChunks; ++i)
            take(order[i], max_batch_rays);
        take(order[0], max_batch_rays);
    }
    if (involved.empty()) return;
    for (uint64_t t : involved) cudaStreamWaitEvent(compute, reqs[t]->h2d, 0);
    if (nch > 0) {
        int flags = 0;
        for (int c = 0; c < nch; ++c) flags |= (H[c].sc.env ? 1 : 0) | (H[c].sc.vox ? 2 : 0);
        cudaMemcpyAsync(chunk_dev[slot], H, sizeof(BakeChunk) * (size_t)nch, cudaMemcpyHostToDevice, compute);
        fipt_status st;
        if (fail_after == 0) {          // injected by fipt_server_inject_launch_failure
            st = fipt_set_error(FIPT_ERR_CUDA, "injected launch failure");
        } else {
            st = launch_bake_batch(chunk_dev[slot], nch, warps, status, compute, flags);
        }
        if (fail_after >= 0) --fail_after;
        if (st != FIPT_OK) set_fatal(st, next_batch, fipt_last_error());
    }
    for (uint64_t t : involved) {
        Req* q = reqs[t];
        if (q->r.kind == FIPT_REQ_RENDER) {
            const Table& tb = tables[q->r.target];
            const int64_t f = q->r.first;
            const size_t row = (size_t)f;
            const float* Ld = tb.Ld + row * 3;
            const float* Ls0 = tb.Ls0 + row * tb.K * 3;
            const float* Ls1 = tb.Ls1 + row * tb.K * 3;
            fipt_status st = fipt_render_fwd(Ld, Ls0, Ls1, q->r.n, tb.K, tb.grid, q->da, q->dr, q->dm,
                                             q->dLgt, nullptr, q->dLr, q->dloss, q->dws, q->ws_bytes,
                                             compute);
            if (st == FIPT_OK)
                st = fipt_render_bwd(Ld, Ls0, Ls1, q->r.n, tb.K, tb.grid, q->da, q->dr, q->dm, q->dLgt,
                                     nullptr, nullptr, q->dga, q->dgr, q->dgm, compute);
            if (st != FIPT_OK) q->result = st;
            q->state = LAUNCHED;
            finishing.push_back(t);
        } else if (q->next >= q->r.n) {
            q->state = LAUNCHED;
            finishing.push_back(t);
        }
    }
    // the batch's device status word lands in this slot's pinned copy
    cudaMemcpyAsync(status_host + slot, status, sizeof(int32_t), cudaMemcpyDeviceToHost, compute);
    cudaMemsetAsync(status, 0, sizeof(int32_t), compute);
    Batch b;
    b.seq = next_batch++;
    b.slot = slot;
    cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    cudaEventRecord(b.done, compute);
    b.finishing = finishing;
    for (uint64_t t : finishing) reqs[t]->last_batch = b.seq;
    inflight.push_back(b);
    active.erase(std::remove_if(active.begin(), active.end(),
                                [&](uint64_t t) { return reqs[t]->state == LAUNCHED; }),
                 active.end());
    ++n_batches;
    n_chunks += (uint64_t)nch;
    rays += (uint64_t)batch_rays;
    max_reqs_in_batch = std::max<uint64_t>(max_reqs_in_batch, involved.size());
}

void fipt_server::retire(Batch& b) {
    const int32_t dev_bits = status_host[b.slot];
    for (uint64_t t : b.finishing) {
        Req* q = reqs[t];
        if (dev_bits != 0 && q->result == FIPT_OK) q->result = FIPT_ERR_DEVICE_CHECK;
        cudaStreamWaitEvent(copy, b.done, 0);
        const size_t n = (size_t)q->r.n;
        if (q->r.kind == FIPT_REQ_BAKE) {
            const size_t K = (size_t)q->r.params.K;
            if (n) {
                cudaMemcpyAsync(q->r.Ld, q->dLd, n * 12, cudaMemcpyDeviceToHost, copy);
                cudaMemcpyAsync(q->r.Ls0, q->dLs0, n * K * 12, cudaMemcpyDeviceToHost, copy);
                cudaMemcpyAsync(q->r.Ls1, q->dLs1, n * K * 12, cudaMemcpyDeviceToHost, copy);
            }
        } else if (n) {
            if (q->r.Lr) cudaMemcpyAsync(q->r.Lr, q->dLr, n * 12, cudaMemcpyDeviceToHost, copy);
            if (q->r.loss) cudaMemcpyAsync(q->r.loss, q->dloss, 8, cudaMemcpyDeviceToHost, copy);
            if (q->r.g_albedo) cudaMemcpyAsync(q->r.g_albedo, q->dga, n * 12, cudaMemcpyDeviceToHost, copy);
            if (q->r.g_rough) cudaMemcpyAsync(q->r.g_rough, q->dgr, n * 4, cudaMemcpyDeviceToHost, copy);
            if (q->r.g_metal) cudaMemcpyAsync(q->r.g_metal, q->dgm, n * 4, cudaMemcpyDeviceToHost, copy);
        }
        cudaEventRecord(q->d2h, copy);
        q->state = COPYING;
        copying.push_back(t);
    }
    cudaEventDestroy(b.done);
}

void fipt_server::finish_copies() {
    for (size_t i = 0; i < copying.size();) {
        Req* q = reqs[copying[i]];
        if (cudaEventQuery(q->d2h) == cudaSuccess) {
            arena->release(q->off, q->bytes);
            q->state = DONE;
            q->t_done = now_s();
            copying.erase(copying.begin() + (long)i);
            cv_done.notify_all();
        } else {
            ++i;
        }
    }
}

void fipt_server::set_fatal(fipt_status st, uint64_t batch, const char* msg) {
    if (fatal != FIPT_OK) return;
    fatal = st;
    fatal_batch = batch;
    snprintf(fatal_msg, sizeof(fatal_msg), "%s", msg ? msg : "");
}

// After a fatal error no new work starts, and every request ends with that
// error -- but only once nothing of it is still in flight: a request whose
// input copy, batch or output copy is still queued on the device keeps the
// caller's host buffers in use until that work has completed (or failed),
// so it is marked done only then.  Batches before the failing one complete
// normally and their requests keep their own results.
void fipt_server::drain_after_fatal() {
    for (uint64_t t : pending) {
        Req* q = reqs[t];
        q->result = fatal;
        q->state = DONE;
        q->t_done = now_s();
    }
    pending.clear();
    for (size_t i = 0; i < active.size();) {
        Req* q = reqs[active[i]];
        if (cudaEventQuery(q->h2d) == cudaErrorNotReady) { ++i; continue; }
        q->result = fatal;
        q->state = DONE;
        q->t_done = now_s();
        active.erase(active.begin() + (long)i);
    }
    while (!inflight.empty()) {
        Batch& b = inflight.front();
        const cudaError_t e = cudaEventQuery(b.done);
        if (e == cudaErrorNotReady) break;
        if (e == cudaSuccess && b.seq < fatal_batch) {
            retire(b);                   // its requests' copies go out as usual
        } else {
            for (uint64_t t : b.finishing) {
                Req* q = reqs[t];
                q->result = fatal;
                q->state = DONE;
                q->t_done = now_s();
            }
            cudaEventDestroy(b.done);
        }
        inflight.pop_front();
    }
    for (size_t i = 0; i < copying.size();) {
        Req* q = reqs[copying[i]];
        const cudaError_t e = cudaEventQuery(q->d2h);
        if (e == cudaErrorNotReady) { ++i; continue; }
        if (e != cudaSuccess && q->result == FIPT_OK) q->result = fatal;
        q->state = DONE;
        q->t_done = now_s();
        copying.erase(copying.begin() + (long)i);
    }
    cv_done.notify_all();
}

void fipt_server::run() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        if (fatal != FIPT_OK) {
            drain_after_fatal();
            if (stop && pending.empty() && active.empty() && inflight.empty() && copying.empty()) break;
            if (pending.empty() && active.empty() && inflight.empty() && copying.empty())
                cv_work.wait_for(lk, std::chrono::milliseconds(10));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
                lk.lock();
            }
            continue;
        }
        bool progress = false;
        // retire finished batches in order
        while (!inflight.empty()) {
            const cudaError_t e = cudaEventQuery(inflight.front().done);
            if (e == cudaErrorNotReady) break;
            if (e != cudaSuccess) {
                char m[200];
                snprintf(m, sizeof(m), "batch failed: %s", cudaGetErrorString(e));
                set_fatal(FIPT_ERR_CUDA, inflight.front().seq, m);
                break;
            }
            retire(inflight.front());
            inflight.pop_front();
            progress = true;
        }
        finish_copies();
        // admit in arrival order while the arena has room
        while (!pending.empty()) {
            Req* q = reqs[pending.front()];
            if (!admit(q)) break;
            active.push_back(q->ticket);
            pending.pop_front();
            progress = true;
        }
        if ((int)inflight.size() < kSlots && !active.empty()) {
            const uint64_t before = n_batches;
            launch_batch();
            progress = progress || n_batches != before;
        }
        if (stop && pending.empty() && active.empty() && inflight.empty() && copying.empty()) break;
        if (!progress) {
            if (inflight.empty() && copying.empty() && active.empty())
                cv_work.wait_for(lk, std::chrono::milliseconds(50));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
                lk.lock();
            }
        }
    }
}

// ---------------------------------------------------------------- C ABI
extern "C" fipt_status fipt_server_create(fipt_ctx* ctx, size_t hbm_budget, int64_t max_batch_rays,
                                          int64_t chunk_points, fipt_server** out) {
    FIPT_REQUIRE(ctx && out, "ctx / out is NULL");
    FIPT_REQUIRE(hbm_budget >= 4096, "hbm_budget too small");
    FIPT_REQUIRE(max_batch_rays > 0 && chunk_points > 0 && chunk_points < ((int64_t)1 << 31),
                 "max_batch_rays and chunk_points must be positive");
    FIPT_CUDA(cudaSetDevice(ctx->device));
    fipt_server* s = new fipt_server();
    s->ctx = ctx;
    s->budget = hbm_budget & ~size_t(255);
    s->max_batch_rays = max_batch_rays;
    s->chunk_points = chunk_points;
    cudaError_t e = cudaMalloc(&s->arena_dev, s->budget);
    if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&s->status_host, sizeof(int32_t) * kSlots);
    for (int i = 0; i < kSlots && e == cudaSuccess; ++i) {
        e = cudaMalloc(&s->chunk_dev[i], sizeof(BakeChunk) * kMaxChunks);
        if (e == cudaSuccess) e = cudaMallocHost(&s->chunk_host[i], sizeof(BakeChunk) * kMaxChunks);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        fipt_server_destroy(s);
        return fipt_check_cuda(e, "server create");
    }
    s->arena = new fipt_arena(s->budget);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_add_scene(fipt_server* s, fipt_scene* scene, int32_t* id) {
    FIPT_REQUIRE(s && scene && id, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->scenes.push_back(scene);
    *id = (int32_t)s->scenes.size() - 1;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_add_table(fipt_server* s, const float* Ld, const float* Ls0,
                                             const float* Ls1, int64_t N, int32_t K,
                                             const float* sigma_grid, int32_t* id) {
    FIPT_REQUIRE(s && id && Ld && Ls0 && Ls1 && sigma_grid, "NULL argument");
    FIPT_REQUIRE(N >= 0 && K >= 2 && K <= FIPT_MAX_K, "bad table size");
    Table t;
    t.Ld = Ld; t.Ls0 = Ls0; t.Ls1 = Ls1; t.N = N; t.K = K;
    for (int k = 0; k < FIPT_MAX_K; ++k) t.grid[k] = k < K ? sigma_grid[k] : sigma_grid[K - 1];
    std::lock_guard<std::mutex> lk(s->mu);
    s->tables.push_back(t);
    *id = (int32_t)s->tables.size() - 1;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_submit(fipt_server* s, const fipt_request* r, uint64_t* ticket) {
    FIPT_REQUIRE(s && r && ticket, "NULL argument");
    FIPT_REQUIRE(r->n >= 0 && r->n < ((int64_t)1 << 31), "bad request size");
    std::unique_lock<std::mutex> lk(s->mu);
    if (r->kind == FIPT_REQ_BAKE) {
        FIPT_REQUIRE(r->target >= 0 && r->target < (int32_t)s->scenes.size(), "unknown scene %d",
                     r->target);
        FIPT_REQUIRE(r->params.K >= 1 && r->params.K <= FIPT_MAX_K && r->params.spp_diffuse >= 1 &&
                     r->params.spp_specular >= 1 && r->params.stats == nullptr,
                     "bad bake parameters (K, spp, stats must be NULL)");
        for (int k = 0; k < r->params.K; ++k)
            FIPT_REQUIRE(r->params.sigma[k] > 0.0f && r->params.sigma[k] <= 1.0f, "sigma out of (0, 1]");
        FIPT_REQUIRE(r->n == 0 || (r->queries && r->Ld && r->Ls0 && r->Ls1), "NULL host buffer");
    } else if (r->kind == FIPT_REQ_RENDER) {
        FIPT_REQUIRE(r->target >= 0 && r->target < (int32_t)s->tables.size(), "unknown table %d",
                     r->target);
        const Table& t = s->tables[r->target];
        FIPT_REQUIRE(r->first >= 0 && r->first + r->n <= t.N, "rows outside the table");
        FIPT_REQUIRE(r->n == 0 || (r->albedo && r->rough && r->metal && r->Lgt), "NULL host buffer");
    } else {
        return fipt_set_error(FIPT_ERR_INVALID_ARG, "unknown request kind %d", r->kind);
    }
    Req* q = new Req();
    q->ticket = s->next_ticket++;
    q->r = *r;
    q->t_submit = now_s();
    q->bytes = request_bytes(*r, s);
    cudaSetDevice(s->ctx->device);
    cudaEventCreateWithFlags(&q->h2d, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&q->d2h, cudaEventDisableTiming);
    s->reqs[q->ticket] = q;
    *ticket = q->ticket;
    if (q->bytes > s->budget) {
        q->state = DONE;
        q->result = FIPT_ERR_BUDGET;
        q->t_done = now_s();
        s->cv_done.notify_all();
        return FIPT_OK;
    }
    s->pending.push_back(q->ticket);
    s->cv_work.notify_one();
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_poll(fipt_server* s, uint64_t ticket, int32_t* done,
                                        fipt_status* result) {
    FIPT_REQUIRE(s && done, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fipt_set_error(FIPT_ERR_NOT_FOUND, "unknown ticket %llu",
                                                   (unsigned long long)ticket);
    *done = it->second->state == DONE;
    if (result) *result = it->second->result;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_wait(fipt_server* s, uint64_t ticket, int64_t timeout_us,
                                        fipt_status* result) {
    FIPT_REQUIRE(s, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fipt_set_error(FIPT_ERR_NOT_FOUND, "unknown ticket %llu",
                                                   (unsigned long long)ticket);
    Req* q = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    while (q->state != DONE) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != DONE)
            return fipt_set_error(FIPT_ERR_TIMEOUT, "request %llu not done after %lld us",
                                  (unsigned long long)ticket, (long long)timeout_us);
    }
    if (result) *result = q->result;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_times(fipt_server* s, uint64_t ticket, double* t_submit,
                                         double* t_admit, double* t_done) {
    FIPT_REQUIRE(s, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fipt_set_error(FIPT_ERR_NOT_FOUND, "unknown ticket");
    if (t_submit) *t_submit = it->second->t_submit;
    if (t_admit) *t_admit = it->second->t_admit;
    if (t_done) *t_done = it->second->t_done;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_release(fipt_server* s, uint64_t ticket) {
    FIPT_REQUIRE(s, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fipt_set_error(FIPT_ERR_NOT_FOUND, "unknown ticket");
    FIPT_REQUIRE(it->second->state == DONE, "request still running");
    cudaEventDestroy(it->second->h2d);
    cudaEventDestroy(it->second->d2h);
    delete it->second;
    s->reqs.erase(it);
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_inject_launch_failure(fipt_server* s, int64_t after_batches) {
    FIPT_REQUIRE(s && after_batches >= 0, "bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    s->fail_after = after_batches;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_get_stats(fipt_server* s, fipt_server_stats* out) {
    FIPT_REQUIRE(s && out, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->batches = s->n_batches;
    out->chunks = s->n_chunks;
    out->rays = s->rays;
    out->max_requests_per_batch = s->max_reqs_in_batch;
    out->bytes_in_use = s->arena ? s->arena->used : 0;
    out->peak_bytes = s->arena ? s->arena->peak : 0;
    out->pending = s->pending.size();
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_destroy(fipt_server* s) {
    if (!s) return FIPT_OK;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
            // requests not yet admitted are cancelled; admitted work drains
            for (uint64_t t : s->pending) {
                Req* q = s->reqs[t];
                q->state = DONE;
                q->result = FIPT_ERR_NOT_FOUND;
            }
            s->pending.clear();
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    cudaSetDevice(s->ctx ? s->ctx->device : 0);
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto& kv : s->reqs) {
        cudaEventDestroy(kv.second->h2d);
        cudaEventDestroy(kv.second->d2h);
        delete kv.second;
    }
    for (int i = 0; i < kSlots; ++i) {
        cudaFree(s->chunk_dev[i]);
        cudaFreeHost(s->chunk_host[i]);
    }
    cudaFreeHost(s->status_host);
    cudaFree(s->status);
    cudaFree(s->arena_dev);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s->arena;
    delete s;
    return FIPT_OK;
}
