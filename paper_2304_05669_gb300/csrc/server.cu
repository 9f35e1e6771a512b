// Serving runtime: device-resident request loops for bakes and renders,
// with continuous batching over several resident scenes on one GPU.
//
//  * Admission.  The server owns one device arena of `hbm_budget` bytes.  A
//    request is admitted (in arrival order) when its device buffers fit in
//    the arena; one larger than the whole budget completes at once with
//    FIPT_ERR_BUDGET.  Inputs are copied in on a copy stream.
//  * The bake loop.  One kernel (k_serve_bake) keeps warps resident on all
//    block slots of every SM but kRenderBlocksPerSM; they take warp items
//    (32 points of one chunk, one lobe) from a device counter in the order
//    the host publishes them and bake each exactly as a standalone
//    fipt_bake would (chunks keep request-local Philox counters), so a
//    result is bit-identical alone and in any mix.  The warp that finishes
//    a chunk raises its flag in host-mapped memory.
//  * The render loop.  A second kernel (k_serve_render) on the remaining
//    block slots takes render items (512 rows of one request) as soon as
//    they are published and computes k_render_fwd_grad's values and loss
//    partials; the warp that finishes a request sums its loss in the render
//    kernels' order.  It is a kernel of its own because render code inside
//    the bake loop cost the bake walk 7 % through register allocation.
//  * Both loops end as a whole: the scheduler stops each (its own flag)
//    after a millisecond without work or on failure, and starts it again
//    when new work is published; a bake warp that waits about half a second
//    in vain ends the bake launch, a render warp that finds no render work
//    for as long ends the render launch.
//  * Continuous batching.  The scheduler thread keeps bake items published
//    ahead of the loop and not yet taken -- two per resident warp, and at
//    least `max_batch_rays` rays -- in chunks of up to `chunk_points`
//    points: the oldest admitted request first, up to a quarter of that,
//    then the requests with the least remaining work, then the oldest
//    again.  A request that arrives while others run has its chunks
//    published as soon as its inputs are on the device, and its warp items
//    interleave with theirs without a new launch.  Render requests are
//    published whole as soon as they are admitted.
//  * Completion.  When a request's last chunk is done, its outputs are
//    copied back on an output stream and its arena space is freed.
//  * All waits are bounded: the scheduler polls events and flags on the
//    host, and the loops' warps give up after a bounded number of polls.
//  * Failure.  A launch that fails, a descriptor copy that fails, or device
//    work that fails stops the server: the loops are told to stop, no new
//    work starts, and every unfinished request ends with that error once
//    none of its copies or kernels is still queued.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <cmath>
#include <vector>

#include "fipt_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kQueue = 1 << 16;          // chunk descriptors per queue epoch
static_assert(kQueue < (1 << FIPT_PUB_CHUNK_BITS), "descriptor count must fit beside the item count");
constexpr int kWaitPolls = 1 << 14;     // naps (about half a second) before a waiting warp ends the launch
constexpr double kIdleStop = 1e-3;       // seconds the loops may idle before the scheduler stops them
constexpr int kRenderBlocksPerSM = 2;    // block slots per SM of the render loop (the bake loop has the rest)
constexpr size_t kOrderPool = (size_t)64 << 20;   // pinned bytes for bake orders on their way to the device
constexpr int64_t kOrderMin = 64;        // smaller bakes keep their own order

// Bit k of a 10-bit value to bit 3k.
uint32_t spread3_10_host(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// The order fipt_query_order gives, on the host: the indices of the points
// sorted (stably) by the 30-bit Morton code of their positions in the box
// [lo, hi]; three 10-bit LSD radix passes, each split over up to eight
// threads (per-thread histograms, then each thread scatters its own range
// after all earlier ranges, which keeps the sort stable).  Served bakes take
// their points in this order so that a warp's points lie together (a
// point's random numbers and outputs use its own index).
void host_query_order(const fipt_query* q, int64_t n, const float lo[3], const float hi[3], int32_t* out) {
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>({8, (int64_t)std::thread::hardware_concurrency(),
                                                              n / 65536}));
    std::vector<uint32_t> key((size_t)n), key2((size_t)n);
    std::vector<int32_t> idx2((size_t)n);
    auto range = [&](int t, int64_t* b, int64_t* e) {
        *b = n * t / T;
        *e = n * (t + 1) / T;
    };
    auto parallel = [&](auto&& fn) {
        std::vector<std::thread> th;
        for (int t = 1; t < T; ++t) th.emplace_back(fn, t);
        fn(0);
        for (auto& x : th) x.join();
    };
    parallel([&](int t) {
        int64_t b, e;
        range(t, &b, &e);
        for (int64_t i = b; i < e; ++i) {
            uint32_t k = 0;
            for (int a = 0; a < 3; ++a) {
                const float ext = hi[a] - lo[a];
                const float u = ext > 0.0f ? (q[i].x[a] - lo[a]) / ext : 0.0f;
                const float c = std::fmin(std::fmax(u * 1024.0f, 0.0f), 1023.0f);
                k |= spread3_10_host((uint32_t)c) << a;
            }
            key[(size_t)i] = k;
            out[i] = (int32_t)i;
        }
    });
    std::vector<int64_t> count((size_t)T * 1024);
    uint32_t* ks = key.data();
    uint32_t* kd = key2.data();
    int32_t* is = out;
    int32_t* id = idx2.data();
    for (int pass = 0; pass < 3; ++pass) {
        const int sh = 10 * pass;
        parallel([&](int t) {
            int64_t b, e;
            range(t, &b, &e);
            int64_t* c = count.data() + (size_t)t * 1024;
            std::fill(c, c + 1024, 0);
            for (int64_t i = b; i < e; ++i) ++c[(ks[i] >> sh) & 1023u];
        });
        int64_t run = 0;                           // offsets: digit-major, thread-minor
        for (int d = 0; d < 1024; ++d)
            for (int t = 0; t < T; ++t) {
                const int64_t c = count[(size_t)t * 1024 + d];
                count[(size_t)t * 1024 + d] = run;
                run += c;
            }
        parallel([&](int t) {
            int64_t b, e;
            range(t, &b, &e);
            int64_t* c = count.data() + (size_t)t * 1024;
            for (int64_t i = b; i < e; ++i) {
                const int64_t d = c[(ks[i] >> sh) & 1023u]++;
                kd[d] = ks[i];
                id[d] = is[i];
            }
        });
        std::swap(ks, kd);
        std::swap(is, id);
    }
    if (is != out) std::memcpy(out, is, sizeof(int32_t) * (size_t)n);
}

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
    int64_t next = 0;             // bake: next slot of its order not yet in a chunk
    int64_t order_off = -1;       // bake: its order in the pinned order pool, or -1 (points in given order)
    int32_t* dorder = nullptr;    // bake: that order on the device
    int chunks_open = 0;          // bake: chunks staged and not yet done
    cudaEvent_t h2d = nullptr, d2h = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Publish {
    cudaEvent_t ev;      // recorded after the publication's copies
    long long warps;     // bake items published once it has landed (-1: a render publication)
};

}  // namespace

struct fipt_server {
    fipt_ctx* ctx = nullptr;
    size_t budget = 0;
    int64_t lookahead_rays = 0, chunk_points = 0;
    int64_t lookahead_items = 0;               // warp items kept published and not yet taken
    int loop_blocks_per_sm = 0;                // resident bake-loop blocks per SM
    int32_t* zero_host = nullptr;              // pinned 0, copied to device flags by the copy engines
    char* arena_dev = nullptr;
    fipt_arena* arena = nullptr;
    cudaStream_t loop = nullptr, loop_r = nullptr, copy = nullptr, d2h = nullptr;
    int32_t* status = nullptr;                 // device status word of this server
    int32_t* status_host = nullptr;            // pinned snapshot, copied with each request's outputs
    // the resident loop's queue
    ServeShared* sh = nullptr;                 // host-mapped control block
    ServeShared* sh_dev = nullptr;
    int32_t* flag_host = nullptr;              // host-mapped per-chunk done flags
    int32_t* flag_dev = nullptr;
    BakeChunk* q_dev = nullptr;                // descriptors on the device
    BakeChunk* q_host = nullptr;               // pinned staging (each slot written once per epoch)
    long long* pub_host = nullptr;             // pinned values of ctr->pub, one per publication this epoch
    int n_pub = 0;
    long long published = 0;                   // warp items whose publication has landed
    ServeCounters* ctr = nullptr;              // device counters of the loop
    long long* orphans[2] = {};                // items a launch leaves to the next one (ping-pong)
    int orphan_parity = 0;
    int32_t* done_dev = nullptr;               // warp items done per chunk
    int n_staged = 0;                          // descriptors staged this epoch
    long long warps_staged = 0;
    std::vector<uint64_t> chunk_req;           // owner of each staged chunk
    std::vector<int64_t> chunk_rays;
    std::vector<int64_t> chunk_items;
    std::vector<long long> chunk_begin;        // first warp item of each staged chunk
    size_t first_untaken = 0;                  // first chunk with items the loop has not taken
    long long taken_seen = 0;                  // most warp items the loop was seen to have taken
    std::vector<int> open_chunks;              // staged, not yet done
    // the render queue (one chunk per render request)
    RenderChunk* r_dev = nullptr;
    RenderChunk* r_host = nullptr;             // pinned staging
    long long* pubr_host = nullptr;            // pinned values of ctr->pub_r
    int32_t* rflag_host = nullptr;             // host-mapped per-chunk done flags
    int32_t* rflag_dev = nullptr;
    int32_t* rdone_dev = nullptr;              // render items done per chunk
    int n_rstaged = 0, n_rpub = 0;
    long long ritems_staged = 0;
    bool published_r = false;                  // a render publication of this epoch has landed
    std::vector<uint64_t> rchunk_req;          // owner of each staged render chunk
    std::vector<int> open_rchunks;
    std::deque<Publish> publishes;             // descriptor copies not yet published
    cudaEvent_t loop_done = nullptr, loop_r_done = nullptr, copy_mark = nullptr;
    bool loop_running = false, loop_r_running = false;
    double idle_since = -1.0;                  // when the running loop last ran out of work
    std::vector<fipt_scene*> scenes;
    std::vector<SceneConst> scene_box;         // host copies of the scenes' constants (bounding box)
    char* order_pool = nullptr;                // pinned: bake orders until their copy to the device lands
    fipt_arena* order_arena = nullptr;         // its bookkeeping
    std::vector<uint64_t> order_staged;        // requests holding a part of the pool
    std::vector<Table> tables;
    std::map<uint64_t, Req*> reqs;
    std::deque<uint64_t> pending;              // arrival order
    std::vector<uint64_t> active;              // admitted bakes with points not yet staged (admission order)
    std::deque<uint64_t> renders;              // admitted render requests not yet staged
    std::vector<uint64_t> copying;
    uint64_t next_ticket = 1;
    // statistics
    uint64_t n_launches = 0, n_chunks = 0, max_reqs_open = 0, rays = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    fipt_status fatal = FIPT_OK;
    int64_t fail_after = -1;                   // test hook: stagings left before an injected failure
    int64_t fail_copy_after = -1;              // test hook: request copy steps left before a refused one
    char fatal_msg[256] = "";

    void run();
    bool admit(Req* q);
    void stage_renders();
    void complete_empty_render(Req* q);
    void stage_chunks();
    void untaken(int64_t* items, int64_t* rays);
    void publish_landed();
    void collect_chunks();
    void retire(Req* q);
    void finish_copies();
    void maybe_reset_epoch();
    void launch_loop();
    void launch_render_loop();
    void stop_idle_loop();
    void release_orders();
    void drain_after_fatal();
    void set_fatal(fipt_status st, const char* msg);
};

namespace {

size_t request_bytes(const fipt_request& r, const fipt_server* s) {
    if (r.kind == FIPT_REQ_BAKE) {
        const size_t n = (size_t)r.n, K = (size_t)r.params.K;
        return up256(n * sizeof(fipt_query)) + up256(n * 3 * 4) + 2 * up256(n * K * 3 * 4) + up256(n * 4) + 256;
    }
    size_t ws = 0;
    fipt_render_workspace_size(r.n, &ws);
    const size_t n = (size_t)r.n;
    (void)s;
    return 4 * up256(n * 12) + 4 * up256(n * 4) + up256(n * 12) + up256(8) + up256(ws) + 256;
}

int64_t rays_per_point(const fipt_bake_params& P) {
    return P.spp_diffuse + (int64_t)P.K * P.spp_specular;
}

}  // namespace

// The first error of a request's copy calls (a refused copy enqueues
// nothing and leaves no sticky error; the thread's last error is cleared so
// that the next launch check does not take it for its own).
static void note_copy(cudaError_t e, cudaError_t* first) {
    if (e == cudaSuccess) return;
    if (*first == cudaSuccess) *first = e;
    cudaGetLastError();
}

// One request's input or output copies were refused: the request ends with
// FIPT_ERR_CUDA (the server goes on) once what it did enqueue is done.
static bool copy_step_fails(int64_t* fail_copy_after, cudaError_t ce) {
    if (*fail_copy_after >= 0 && (*fail_copy_after)-- == 0) return true;   // injected
    return ce != cudaSuccess;
}

bool fipt_server::admit(Req* q) {
    size_t off;
    if (!arena->alloc(q->bytes, &off)) return false;
    q->off = off;
    q->base = arena_dev + off;
    Carver c{q->base, 0};
    const fipt_request& r = q->r;
    const size_t n = (size_t)r.n;
    cudaError_t ce = cudaSuccess;
    if (r.kind == FIPT_REQ_BAKE) {
        const size_t K = (size_t)r.params.K;
        q->dq = c.take<fipt_query>(n);
        q->dLd = c.take<float>(n * 3);
        q->dLs0 = c.take<float>(n * K * 3);
        q->dLs1 = c.take<float>(n * K * 3);
        q->dorder = c.take<int32_t>(n);
        if (n) note_copy(cudaMemcpyAsync(q->dq, r.queries, n * sizeof(fipt_query), cudaMemcpyHostToDevice, copy), &ce);
        if (q->order_off >= 0)
            note_copy(cudaMemcpyAsync(q->dorder, order_pool + q->order_off, n * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, copy), &ce);
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
            note_copy(cudaMemcpyAsync(q->da, r.albedo, n * 12, cudaMemcpyHostToDevice, copy), &ce);
            note_copy(cudaMemcpyAsync(q->dr, r.rough, n * 4, cudaMemcpyHostToDevice, copy), &ce);
            note_copy(cudaMemcpyAsync(q->dm, r.metal, n * 4, cudaMemcpyHostToDevice, copy), &ce);
            note_copy(cudaMemcpyAsync(q->dLgt, r.Lgt, n * 12, cudaMemcpyHostToDevice, copy), &ce);
        }
    }
    note_copy(cudaEventRecord(q->h2d, copy), &ce);
    if (copy_step_fails(&fail_copy_after, ce)) q->result = FIPT_ERR_CUDA;
    q->state = ADMITTED;
    q->t_admit = now_s();
    return true;
}

// Publishes the admitted render requests, one chunk each.  The loop takes
// a render item before any bake item, so a render request starts as soon
// as warps finish the items they hold.  Its descriptor goes to the device
// on the copy stream after its input copies.
void fipt_server::stage_renders() {
    const int first = n_rstaged;
    while (!renders.empty() && n_rstaged < kQueue) {
        Req* q = reqs[renders.front()];
        renders.pop_front();
        const Table& tb = tables[q->r.target];
        const size_t row = (size_t)q->r.first;
        RenderChunk& C = r_host[n_rstaged];
        C.Ld = tb.Ld + row * 3;
        C.Ls0 = tb.Ls0 + row * tb.K * 3;
        C.Ls1 = tb.Ls1 + row * tb.K * 3;
        C.albedo = q->da;
        C.rough = q->dr;
        C.metal = q->dm;
        C.Lgt = q->dLgt;
        C.Lr = q->dLr;
        C.g_albedo = q->dga;
        C.g_rough = q->dgr;
        C.g_metal = q->dgm;
        C.partial = static_cast<double*>(q->dws);
        C.loss = q->dloss;
        C.n = q->r.n;
        C.item_begin = ritems_staged;
        C.K = tb.K;
        for (int k = 0; k < FIPT_MAX_K; ++k) C.grid[k] = tb.grid[k];
        ritems_staged += (q->r.n + FIPT_RENDER_ITEM_ROWS - 1) / FIPT_RENDER_ITEM_ROWS;
        rchunk_req.push_back(q->ticket);
        open_rchunks.push_back(n_rstaged);
        q->state = LAUNCHED;
        ++n_rstaged;
    }
    const int count = n_rstaged - first;
    if (count == 0) return;
    if (fail_after >= 0 && fail_after-- == 0) {    // injected by fipt_server_inject_launch_failure
        set_fatal(FIPT_ERR_CUDA, "injected launch failure");
        return;
    }
    cudaError_t ce = cudaSuccess;
    note_copy(cudaMemcpyAsync(r_dev + first, r_host + first, sizeof(RenderChunk) * (size_t)count,
                              cudaMemcpyHostToDevice, copy), &ce);
    pubr_host[n_rpub] = (ritems_staged << FIPT_PUB_CHUNK_BITS) | n_rstaged;
    note_copy(cudaMemcpyAsync(&ctr->pub_r, pubr_host + n_rpub, sizeof(long long), cudaMemcpyHostToDevice, copy),
              &ce);
    ++n_rpub;
    Publish p{};
    note_copy(cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming), &ce);
    if (ce == cudaSuccess) note_copy(cudaEventRecord(p.ev, copy), &ce);
    if (ce != cudaSuccess) {
        if (p.ev) cudaEventDestroy(p.ev);
        set_fatal(FIPT_ERR_CUDA, "render descriptor copy failed");
        return;
    }
    p.warps = -1;
    publishes.push_back(p);
}

// A render request of no rows: its loss is 0 and nothing runs.
void fipt_server::complete_empty_render(Req* q) {
    if (q->r.loss) *q->r.loss = 0.0;
    arena->release(q->off, q->bytes);
    q->state = DONE;
    q->t_done = now_s();
    cv_done.notify_all();
}

// Warp items (and their rays) staged but not yet taken by the loop.  The
// loop's warps take items in staging order, so everything below the taken
// mark is taken; the mark the warps write is a recent one, not always the
// highest, so the scheduler keeps the highest it has seen.
void fipt_server::untaken(int64_t* items, int64_t* rays) {
    taken_seen = std::max(taken_seen, __atomic_load_n(&sh->taken, __ATOMIC_RELAXED));
    const long long t = std::min<long long>(taken_seen, warps_staged);
    while (first_untaken < chunk_begin.size() &&
           chunk_begin[first_untaken] + chunk_items[first_untaken] <= t)
        ++first_untaken;
    int64_t r = 0;
    for (size_t c = first_untaken; c < chunk_begin.size(); ++c) {
        const long long from = std::max<long long>(chunk_begin[c], t);
        r += (int64_t)((double)chunk_rays[c] * (double)(chunk_begin[c] + chunk_items[c] - from) / (double)chunk_items[c]);
    }
    *items = warps_staged - t;
    *rays = r;
}

// Stages chunk descriptors while fewer than lookahead_items warp items (two
// per resident warp of the loop) and fewer than lookahead_rays rays are
// published and not yet taken: the oldest admitted bake first, up to a
// quarter of lookahead_items, then the bakes with the least remaining work,
// then the oldest again.  Counting items not yet taken (rather than items
// not yet done) keeps the loop fed while a chunk's last items run long.
// The new descriptors go to the device on the copy stream (after the
// requests' input copies) and are published once that copy has landed.
void fipt_server::stage_chunks() {
    int64_t items_ahead = 0, rays_ahead = 0;
    untaken(&items_ahead, &rays_ahead);
    if (n_staged >= kQueue || (items_ahead >= lookahead_items && rays_ahead >= lookahead_rays)) return;
    std::vector<uint64_t> order;
    for (uint64_t t : active) order.push_back(t);
    if (order.empty()) return;
    auto remaining = [&](uint64_t t) {
        const Req* q = reqs[t];
        return (q->r.n - q->next) * rays_per_point(q->r.params);
    };
    if (order.size() > 1)
        std::stable_sort(order.begin() + 1, order.end(),
                         [&](uint64_t a, uint64_t b) { return remaining(a) < remaining(b); });
    const int first = n_staged;
    auto take = [&](uint64_t t, int64_t share) {
        Req* q = reqs[t];
        const fipt_bake_params& P = q->r.params;
        const int64_t rpp = rays_per_point(P);
        int64_t got = 0;
        while (q->next < q->r.n && n_staged < kQueue) {
            const int64_t c = std::min<int64_t>(chunk_points, q->r.n - q->next);
            const int64_t items = ((c + 31) / 32) * (1 + P.K);
            const bool full = items_ahead + items > lookahead_items && rays_ahead + c * rpp > lookahead_rays;
            if (items_ahead > 0 && (full || got + items > share)) break;
            BakeChunk& C = q_host[n_staged];
            fipt_scene* sc = scenes[q->r.target];
            C.sc = sc->view();
            if (q->order_off >= 0) {            // slots of the order: the request's own indices
                C.q = q->dq;
                C.Ld = q->dLd;
                C.Ls0 = q->dLs0;
                C.Ls1 = q->dLs1;
                C.order = q->dorder + q->next;
            } else {
                C.q = q->dq + q->next;
                C.Ld = q->dLd + 3 * q->next;
                C.Ls0 = q->dLs0 + q->next * P.K * 3;
                C.Ls1 = q->dLs1 + q->next * P.K * 3;
                C.order = nullptr;
            }
            C.n = c;
            C.warp_begin = warps_staged;
            C.A.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
            C.A.request_id = P.request_id;
            C.A.point_base = q->order_off >= 0 ? 0u : (uint32_t)q->next;
            C.A.spp_d = P.spp_diffuse;
            C.A.spp_s = P.spp_specular;
            C.A.K = P.K;
            set_strata(C.A);
            for (int k = 0; k < FIPT_MAX_K; ++k) C.A.sigma[k] = k < P.K ? P.sigma[k] : 1.0f;
            chunk_begin.push_back(warps_staged);
            warps_staged += items;
            chunk_req.push_back(t);
            chunk_rays.push_back(c * rpp);
            chunk_items.push_back(items);
            open_chunks.push_back(n_staged);
            items_ahead += items;
            rays_ahead += c * rpp;
            got += items;
            q->next += c;
            ++q->chunks_open;
            ++n_staged;
        }
    };
    const int64_t total = std::max<int64_t>(lookahead_items, 1);
    take(order[0], total / 4);
    for (size_t i = 1; i < order.size() && n_staged < kQueue &&
                       (items_ahead < lookahead_items || rays_ahead < lookahead_rays); ++i)
        take(order[i], INT64_MAX);
    take(order[0], INT64_MAX);
    active.erase(std::remove_if(active.begin(), active.end(),
                                [&](uint64_t t) {
                                    Req* q = reqs[t];
                                    if (q->next < q->r.n) return false;
                                    q->state = LAUNCHED;
                                    return true;
                                }),
                 active.end());
    const int count = n_staged - first;
    if (count == 0) return;
    if (fail_after >= 0 && fail_after-- == 0) {    // injected by fipt_server_inject_launch_failure
        set_fatal(FIPT_ERR_CUDA, "injected launch failure");
        return;
    }
    cudaError_t ce = cudaSuccess;
    note_copy(cudaMemcpyAsync(q_dev + first, q_host + first, sizeof(BakeChunk) * (size_t)count,
                              cudaMemcpyHostToDevice, copy), &ce);
    // then the count the loop polls, behind the descriptors on the same stream
    pub_host[n_pub] = ((long long)warps_staged << FIPT_PUB_CHUNK_BITS) | n_staged;
    note_copy(cudaMemcpyAsync(&ctr->pub, pub_host + n_pub, sizeof(long long), cudaMemcpyHostToDevice, copy), &ce);
    ++n_pub;
    Publish p{};
    note_copy(cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming), &ce);
    if (ce == cudaSuccess) note_copy(cudaEventRecord(p.ev, copy), &ce);
    if (ce != cudaSuccess) {
        if (p.ev) cudaEventDestroy(p.ev);
        set_fatal(FIPT_ERR_CUDA, "bake descriptor copy failed");
        return;
    }
    p.warps = warps_staged;
    publishes.push_back(p);
    n_chunks += (uint64_t)count;
    uint64_t open_reqs = 0;
    for (auto& kv : reqs)
        if (kv.second->r.kind == FIPT_REQ_BAKE && kv.second->chunks_open > 0) ++open_reqs;
    max_reqs_open = std::max(max_reqs_open, open_reqs);
}

// Notes the publications that have landed (the loop sees each as soon as
// its copy lands; the scheduler's record is for starting the loop).
void fipt_server::publish_landed() {
    while (!publishes.empty()) {
        Publish& p = publishes.front();
        const cudaError_t e = cudaEventQuery(p.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) {
            set_fatal(FIPT_ERR_CUDA, "descriptor copy failed");
            return;
        }
        if (p.warps < 0) published_r = true;
        else published = p.warps;
        cudaEventDestroy(p.ev);
        publishes.pop_front();
    }
}

// Chunks whose flags the loop has raised: a bake request whose last chunk
// is done, and a render request whose chunk is, get their outputs copied
// back.
void fipt_server::collect_chunks() {
    for (size_t i = 0; i < open_chunks.size();) {
        const int c = open_chunks[i];
        if (__atomic_load_n(flag_host + c, __ATOMIC_ACQUIRE) == 0) { ++i; continue; }
        open_chunks[i] = open_chunks.back();
        open_chunks.pop_back();
        rays += (uint64_t)chunk_rays[c];
        Req* q = reqs[chunk_req[c]];
        if (--q->chunks_open == 0 && q->next >= q->r.n) retire(q);
    }
    for (size_t i = 0; i < open_rchunks.size();) {
        const int c = open_rchunks[i];
        if (__atomic_load_n(rflag_host + c, __ATOMIC_ACQUIRE) == 0) { ++i; continue; }
        open_rchunks[i] = open_rchunks.back();
        open_rchunks.pop_back();
        retire(reqs[rchunk_req[c]]);
    }
}

// Copies a finished request's outputs back (with a snapshot of the device
// status word) on the output stream, so they never hold up a publication.
void fipt_server::retire(Req* q) {
    const size_t n = (size_t)q->r.n;
    cudaError_t ce = cudaSuccess;
    if (q->r.kind == FIPT_REQ_BAKE) {
        const size_t K = (size_t)q->r.params.K;
        if (n) {
            note_copy(cudaMemcpyAsync(q->r.Ld, q->dLd, n * 12, cudaMemcpyDeviceToHost, d2h), &ce);
            note_copy(cudaMemcpyAsync(q->r.Ls0, q->dLs0, n * K * 12, cudaMemcpyDeviceToHost, d2h), &ce);
            note_copy(cudaMemcpyAsync(q->r.Ls1, q->dLs1, n * K * 12, cudaMemcpyDeviceToHost, d2h), &ce);
        }
    } else {
        if (n) {
            if (q->r.Lr) note_copy(cudaMemcpyAsync(q->r.Lr, q->dLr, n * 12, cudaMemcpyDeviceToHost, d2h), &ce);
            if (q->r.loss) note_copy(cudaMemcpyAsync(q->r.loss, q->dloss, 8, cudaMemcpyDeviceToHost, d2h), &ce);
            if (q->r.g_albedo)
                note_copy(cudaMemcpyAsync(q->r.g_albedo, q->dga, n * 12, cudaMemcpyDeviceToHost, d2h), &ce);
            if (q->r.g_rough)
                note_copy(cudaMemcpyAsync(q->r.g_rough, q->dgr, n * 4, cudaMemcpyDeviceToHost, d2h), &ce);
            if (q->r.g_metal)
                note_copy(cudaMemcpyAsync(q->r.g_metal, q->dgm, n * 4, cudaMemcpyDeviceToHost, d2h), &ce);
        }
    }
    note_copy(cudaMemcpyAsync(status_host, status, sizeof(int32_t), cudaMemcpyDeviceToHost, d2h), &ce);
    note_copy(cudaEventRecord(q->d2h, d2h), &ce);
    if (copy_step_fails(&fail_copy_after, ce) && q->result == FIPT_OK) q->result = FIPT_ERR_CUDA;
    q->state = COPYING;
    copying.push_back(q->ticket);
}

void fipt_server::finish_copies() {
    for (size_t i = 0; i < copying.size();) {
        Req* q = reqs[copying[i]];
        if (cudaEventQuery(q->d2h) == cudaSuccess) {
            if (*reinterpret_cast<volatile int32_t*>(status_host) != 0 && q->result == FIPT_OK)
                q->result = FIPT_ERR_DEVICE_CHECK;
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

// Starts a new queue epoch once every staged chunk is done and the loop
// has left: counters back to zero on the device and in the mapped block.
void fipt_server::maybe_reset_epoch() {
    if ((n_staged == 0 && n_rstaged == 0) || loop_running || loop_r_running || !open_chunks.empty() ||
        !open_rchunks.empty() || !publishes.empty())
        return;
    std::memset(flag_host, 0, sizeof(int32_t) * (size_t)n_staged);
    std::memset(rflag_host, 0, sizeof(int32_t) * (size_t)n_rstaged);
    // on the copy stream, ahead of the next epoch's publications
    cudaError_t ce = cudaSuccess;
    note_copy(cudaMemsetAsync(ctr, 0, sizeof(ServeCounters), copy), &ce);
    if (n_staged) note_copy(cudaMemsetAsync(done_dev, 0, sizeof(int32_t) * (size_t)n_staged, copy), &ce);
    if (n_rstaged) note_copy(cudaMemsetAsync(rdone_dev, 0, sizeof(int32_t) * (size_t)n_rstaged, copy), &ce);
    if (ce != cudaSuccess) set_fatal(FIPT_ERR_CUDA, "queue reset failed");
    published = 0;
    n_pub = 0;
    published_r = false;
    n_rstaged = 0;
    n_rpub = 0;
    ritems_staged = 0;
    rchunk_req.clear();
    __atomic_store_n(&sh->taken, 0LL, __ATOMIC_RELAXED);
    n_staged = 0;
    warps_staged = 0;
    taken_seen = 0;
    first_untaken = 0;
    chunk_req.clear();
    chunk_rays.clear();
    chunk_items.clear();
    chunk_begin.clear();
}

// Starts the resident loop when it is not running and staged work waits:
// items not yet taken, or items an earlier launch left behind.  It waits
// for the epoch's first publication, so its warps do not spend their idle
// polls on a descriptor copy.
void fipt_server::launch_loop() {
    if (loop_running || open_chunks.empty() || published == 0) return;
    if (fail_after >= 0 && fail_after-- == 0) {
        set_fatal(FIPT_ERR_CUDA, "injected launch failure");
        return;
    }
    int flags = 0;
    for (fipt_scene* sc : scenes) flags |= (sc->env ? 1 : 0) | (sc->vox ? 2 : 0);
    // after the copy stream's counter resets; the previous launch's orphans
    // become this one's inputs
    cudaEventRecord(copy_mark, copy);
    cudaStreamWaitEvent(loop, copy_mark, 0);
    cudaMemcpyAsync(&ctr->n_in, &ctr->n_out, sizeof(int), cudaMemcpyDeviceToDevice, loop);
    cudaMemsetAsync(&ctr->take_in, 0, sizeof(int), loop);
    cudaMemsetAsync(&ctr->n_out, 0, sizeof(int), loop);
    cudaMemsetAsync(&ctr->quit, 0, sizeof(int), loop);
    __atomic_store_n(&sh->stop, 0, __ATOMIC_RELAXED);   // ordered before the launch by the launch itself
    idle_since = -1.0;
    fipt_status st = launch_serve_bake(q_dev, sh_dev, ctr, orphans[orphan_parity], orphans[1 - orphan_parity],
                                       done_dev, flag_dev, status, kWaitPolls, loop_blocks_per_sm, loop, flags);
    orphan_parity ^= 1;
    if (st != FIPT_OK) {
        set_fatal(st, fipt_last_error());
        return;
    }
    cudaEventRecord(loop_done, loop);
    loop_running = true;
    ++n_launches;
}

// Starts the render loop when it is not running and published render work
// waits (its warps leave when they find none for a while).  Its quit flag
// is cleared by a copy, not a memset kernel: the bake loop may hold every
// other block slot.
void fipt_server::launch_render_loop() {
    if (loop_r_running || open_rchunks.empty() || !published_r) return;
    if (fail_after >= 0 && fail_after-- == 0) {
        set_fatal(FIPT_ERR_CUDA, "injected launch failure");
        return;
    }
    cudaEventRecord(copy_mark, copy);
    cudaStreamWaitEvent(loop_r, copy_mark, 0);
    cudaMemcpyAsync(&ctr->quit_r, zero_host, sizeof(int32_t), cudaMemcpyHostToDevice, loop_r);
    // each loop has its own stop flag, cleared only when that loop has left
    // entirely (a bake warp that saw its flag cleared while the others left
    // would stay resident alone)
    __atomic_store_n(&sh->stop_r, 0, __ATOMIC_RELAXED);   // ordered before the launch by the launch itself
    idle_since = -1.0;
    const fipt_status st = launch_serve_render(r_dev, sh_dev, ctr, rdone_dev, rflag_dev, kWaitPolls,
                                               kRenderBlocksPerSM, loop_r);
    if (st != FIPT_OK) {
        set_fatal(st, fipt_last_error());
        return;
    }
    cudaEventRecord(loop_r_done, loop_r);
    loop_r_running = true;
}

// Returns a request's part of the order pool once its copy to the device
// has landed (or the request ended without being admitted).
void fipt_server::release_orders() {
    for (size_t i = 0; i < order_staged.size();) {
        Req* q = reqs[order_staged[i]];
        const bool done = q->state == DONE || (q->state != PENDING && cudaEventQuery(q->h2d) == cudaSuccess);
        if (!done) { ++i; continue; }
        order_arena->release((size_t)q->order_off, (size_t)q->r.n * sizeof(int32_t));
        order_staged[i] = order_staged.back();
        order_staged.pop_back();
    }
}

// Stops the running loops once they have had no work for kIdleStop seconds,
// so their resident blocks do not hold the SMs while the server is idle.
void fipt_server::stop_idle_loop() {
    if ((!loop_running && !loop_r_running) || !open_chunks.empty() || !open_rchunks.empty() ||
        !publishes.empty()) {
        idle_since = -1.0;
        return;
    }
    const double t = now_s();
    if (idle_since < 0.0) idle_since = t;
    else if (t - idle_since > kIdleStop) {
        __atomic_store_n(&sh->stop, 1, __ATOMIC_RELEASE);
        __atomic_store_n(&sh->stop_r, 1, __ATOMIC_RELEASE);
    }
}

void fipt_server::set_fatal(fipt_status st, const char* msg) {
    if (fatal != FIPT_OK) return;
    fatal = st;
    snprintf(fatal_msg, sizeof(fatal_msg), "%s", msg ? msg : "");
    __atomic_store_n(&sh->stop, 1, __ATOMIC_RELEASE);    // the loops leave after the items they hold
    __atomic_store_n(&sh->stop_r, 1, __ATOMIC_RELEASE);
}

// After a fatal error no new work starts, and every unfinished request ends
// with that error -- but only once nothing of it is still in flight: its
// input copy, the loop (which may hold its chunks) and its output copies
// must have completed or failed before the caller may reuse its buffers.
// Requests already copying their outputs keep their own results.
void fipt_server::drain_after_fatal() {
    for (uint64_t t : pending) {
        Req* q = reqs[t];
        q->result = fatal;
        q->state = DONE;
        q->t_done = now_s();
    }
    pending.clear();
    if (loop_running && cudaEventQuery(loop_done) != cudaErrorNotReady) loop_running = false;
    if (loop_r_running && cudaEventQuery(loop_r_done) != cudaErrorNotReady) loop_r_running = false;
    while (!publishes.empty() && cudaEventQuery(publishes.front().ev) != cudaErrorNotReady) {
        cudaEventDestroy(publishes.front().ev);
        publishes.pop_front();
    }
    const bool device_quiet = !loop_running && !loop_r_running && publishes.empty();
    for (auto& kv : reqs) {
        Req* q = kv.second;
        if (q->state == DONE || q->state == COPYING) continue;
        if (!device_quiet) continue;
        if (cudaEventQuery(q->h2d) == cudaErrorNotReady) continue;
        q->result = fatal;
        q->state = DONE;
        q->t_done = now_s();
    }
    if (device_quiet) {
        active.clear();
        renders.erase(std::remove_if(renders.begin(), renders.end(),
                                     [&](uint64_t t) { return reqs[t]->state == DONE; }),
                      renders.end());
        open_chunks.clear();
        open_rchunks.clear();
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
            bool busy = false;
            for (auto& kv : reqs) busy = busy || kv.second->state != DONE;
            if (stop && !busy && !loop_running && !loop_r_running && publishes.empty()) break;
            if (!busy && !loop_running && !loop_r_running)
                cv_work.wait_for(lk, std::chrono::milliseconds(10));
            else {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(50));
                lk.lock();
            }
            continue;
        }
        bool failed = false;
        for (int k = 0; k < 2; ++k) {
            bool& running = k == 0 ? loop_running : loop_r_running;
            if (!running) continue;
            const cudaError_t e = cudaEventQuery(k == 0 ? loop_done : loop_r_done);
            if (e == cudaErrorNotReady) continue;
            running = false;
            if (e != cudaSuccess) {
                char m[200];
                snprintf(m, sizeof(m), "serving loop failed: %s", cudaGetErrorString(e));
                set_fatal(FIPT_ERR_CUDA, m);
                failed = true;
            }
        }
        if (failed) continue;
        publish_landed();
        collect_chunks();
        finish_copies();
        release_orders();
        if (fatal != FIPT_OK) continue;
        // admit in arrival order while the arena has room
        bool admitted = false;
        while (!pending.empty()) {
            Req* q = reqs[pending.front()];
            if (!admit(q)) break;
            pending.pop_front();
            admitted = true;
            if (q->result != FIPT_OK) {     // its input copies were refused: nothing of it runs
                cudaEventRecord(q->d2h, copy);          // after what it did enqueue
                q->state = COPYING;
                copying.push_back(q->ticket);
                continue;
            }
            if (q->r.kind == FIPT_REQ_BAKE) {
                if (q->r.n > 0) active.push_back(q->ticket);
                else retire(q);
            } else if (q->r.n > 0) {
                renders.push_back(q->ticket);
            } else {
                complete_empty_render(q);
            }
        }
        if (fatal != FIPT_OK) continue;
        maybe_reset_epoch();
        stage_renders();
        if (fatal != FIPT_OK) continue;
        stage_chunks();
        if (fatal != FIPT_OK) continue;
        publish_landed();
        launch_render_loop();
        if (fatal != FIPT_OK) continue;
        launch_loop();
        stop_idle_loop();
        const bool idle = pending.empty() && active.empty() && open_chunks.empty() && renders.empty() &&
                          open_rchunks.empty() && copying.empty() && publishes.empty();
        if (stop && idle && !loop_running && !loop_r_running) break;
        if (idle && !admitted && !loop_running && !loop_r_running) {
            cv_work.wait_for(lk, std::chrono::milliseconds(50));
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        }
    }
}

extern "C" fipt_status fipt_server_create(fipt_ctx* ctx, size_t hbm_budget, int64_t max_batch_rays,
                                          int64_t chunk_points, fipt_server** out) {
    FIPT_REQUIRE(ctx && out, "ctx / out is NULL");
    FIPT_REQUIRE(hbm_budget >= 4096, "hbm_budget too small");
    FIPT_REQUIRE(max_batch_rays > 0 && chunk_points > 0 && chunk_points < ((int64_t)1 << 31),
                 "max_batch_rays and chunk_points must be positive");
    FIPT_CUDA(cudaSetDevice(ctx->device));
    // the render loop takes kRenderBlocksPerSM block slots of every SM and
    // the bake loop all the others its registers allow; asking also loads
    // the loops' kernels
    int loop_bps = 0;
    {
        const fipt_status fs = serve_loop_blocks_per_sm(&loop_bps);
        if (fs != FIPT_OK) return fs;
        loop_bps -= kRenderBlocksPerSM;
        FIPT_REQUIRE(loop_bps >= 1, "the serving loops do not fit on an SM");
    }
    fipt_server* s = new fipt_server();
    s->ctx = ctx;
    s->budget = hbm_budget & ~size_t(255);
    s->lookahead_rays = max_batch_rays;
    s->loop_blocks_per_sm = loop_bps;
    s->lookahead_items = 2 * (int64_t)serve_loop_warps(s->loop_blocks_per_sm);
    s->chunk_points = chunk_points;
    cudaError_t e = cudaMalloc(&s->arena_dev, s->budget);
    if (e == cudaSuccess) e = cudaMalloc(&s->status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(s->status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&s->status_host, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaHostAlloc(&s->sh, sizeof(ServeShared), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->sh_dev, s->sh, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->flag_host, sizeof(int32_t) * kQueue, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->flag_dev, s->flag_host, 0);
    if (e == cudaSuccess) e = cudaMalloc(&s->q_dev, sizeof(BakeChunk) * kQueue);
    if (e == cudaSuccess) e = cudaMallocHost(&s->q_host, sizeof(BakeChunk) * kQueue);
    if (e == cudaSuccess) e = cudaMallocHost(&s->pub_host, sizeof(long long) * kQueue);
    if (e == cudaSuccess) e = cudaMalloc(&s->ctr, sizeof(ServeCounters));
    if (e == cudaSuccess) e = cudaMemset(s->ctr, 0, sizeof(ServeCounters));
    const size_t max_orphans = (size_t)serve_loop_warps(s->loop_blocks_per_sm);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaMalloc(&s->orphans[i], sizeof(long long) * max_orphans);
    if (e == cudaSuccess) e = cudaMalloc(&s->done_dev, sizeof(int32_t) * kQueue);
    if (e == cudaSuccess) e = cudaMemset(s->done_dev, 0, sizeof(int32_t) * kQueue);
    if (e == cudaSuccess) e = cudaMalloc(&s->r_dev, sizeof(RenderChunk) * kQueue);
    if (e == cudaSuccess) e = cudaMallocHost(&s->r_host, sizeof(RenderChunk) * kQueue);
    if (e == cudaSuccess) e = cudaMallocHost(&s->pubr_host, sizeof(long long) * kQueue);
    if (e == cudaSuccess) e = cudaMallocHost(&s->order_pool, kOrderPool);
    if (e == cudaSuccess) e = cudaHostAlloc(&s->rflag_host, sizeof(int32_t) * kQueue, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s->rflag_dev, s->rflag_host, 0);
    if (e == cudaSuccess) e = cudaMalloc(&s->rdone_dev, sizeof(int32_t) * kQueue);
    if (e == cudaSuccess) e = cudaMemset(s->rdone_dev, 0, sizeof(int32_t) * kQueue);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->loop, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->loop_r, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&s->zero_host, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->loop_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->copy_mark, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->loop_r_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fipt_server_destroy(s);
        return fipt_check_cuda(e, "server create");
    }
    std::memset(s->sh, 0, sizeof(ServeShared));
    *s->zero_host = 0;
    std::memset(s->flag_host, 0, sizeof(int32_t) * kQueue);
    std::memset(s->rflag_host, 0, sizeof(int32_t) * kQueue);
    s->arena = new fipt_arena(s->budget);
    s->order_arena = new fipt_arena(kOrderPool);
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_add_scene(fipt_server* s, fipt_scene* scene, int32_t* id) {
    FIPT_REQUIRE(s && scene && id, "NULL argument");
    SceneConst box;
    FIPT_CUDA(cudaMemcpy(&box, scene->cst, sizeof(box), cudaMemcpyDeviceToHost));
    std::lock_guard<std::mutex> lk(s->mu);
    s->scenes.push_back(scene);
    s->scene_box.push_back(box);
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
                     r->params.spp_specular >= 1 && r->params.stats == nullptr && r->params.order == nullptr,
                     "bad bake parameters (K, spp; stats and order must be NULL)");
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
    // a bake's points in Morton order of their positions: a part of the
    // pinned order pool (or none when it is full: the points keep their
    // order), filled by this thread outside the lock
    const double t_submit = now_s();
    int64_t order_off = -1;
    if (r->kind == FIPT_REQ_BAKE && r->n >= kOrderMin && request_bytes(*r, s) <= s->budget) {
        size_t off = 0;
        if (s->order_arena->alloc((size_t)r->n * sizeof(int32_t), &off)) {
            order_off = (int64_t)off;
            const SceneConst box = s->scene_box[r->target];
            lk.unlock();
            host_query_order(r->queries, r->n, box.lo, box.hi, reinterpret_cast<int32_t*>(s->order_pool + off));
            lk.lock();
        }
    }
    Req* q = new Req();
    q->ticket = s->next_ticket++;
    q->r = *r;
    q->t_submit = t_submit;
    q->order_off = order_off;
    if (order_off >= 0) s->order_staged.push_back(q->ticket);
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

extern "C" fipt_status fipt_server_inject_launch_failure(fipt_server* s, int64_t after_launches) {
    FIPT_REQUIRE(s && after_launches >= 0, "bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    s->fail_after = after_launches;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_inject_copy_failure(fipt_server* s, int64_t after_steps) {
    FIPT_REQUIRE(s && after_steps >= 0, "bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    s->fail_copy_after = after_steps;
    return FIPT_OK;
}

extern "C" fipt_status fipt_server_get_stats(fipt_server* s, fipt_server_stats* out) {
    FIPT_REQUIRE(s && out, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    out->batches = s->n_launches;
    out->chunks = s->n_chunks;
    out->rays = s->rays;
    out->max_requests_per_batch = s->max_reqs_open;
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
    if (s->sh) {
        __atomic_store_n(&s->sh->stop, 1, __ATOMIC_RELEASE);
        __atomic_store_n(&s->sh->stop_r, 1, __ATOMIC_RELEASE);
    }
    if (s->loop) cudaStreamSynchronize(s->loop);
    if (s->loop_r) cudaStreamSynchronize(s->loop_r);
    if (s->copy) cudaStreamSynchronize(s->copy);
    if (s->d2h) cudaStreamSynchronize(s->d2h);
    for (auto& p : s->publishes) cudaEventDestroy(p.ev);
    for (auto& kv : s->reqs) {
        cudaEventDestroy(kv.second->h2d);
        cudaEventDestroy(kv.second->d2h);
        delete kv.second;
    }
    if (s->loop_done) cudaEventDestroy(s->loop_done);
    if (s->copy_mark) cudaEventDestroy(s->copy_mark);
    if (s->loop_r_done) cudaEventDestroy(s->loop_r_done);
    if (s->zero_host) cudaFreeHost(s->zero_host);
    cudaFree(s->q_dev);
    cudaFreeHost(s->q_host);
    cudaFreeHost(s->pub_host);
    cudaFree(s->ctr);
    cudaFree(s->orphans[0]);
    cudaFree(s->orphans[1]);
    cudaFree(s->done_dev);
    cudaFreeHost(s->flag_host);
    cudaFree(s->r_dev);
    cudaFreeHost(s->r_host);
    cudaFreeHost(s->pubr_host);
    if (s->order_pool) cudaFreeHost(s->order_pool);
    delete s->order_arena;
    cudaFreeHost(s->rflag_host);
    cudaFree(s->rdone_dev);
    cudaFreeHost(s->sh);
    cudaFreeHost(s->status_host);
    cudaFree(s->status);
    cudaFree(s->arena_dev);
    if (s->loop) cudaStreamDestroy(s->loop);
    if (s->loop_r) cudaStreamDestroy(s->loop_r);
    if (s->copy) cudaStreamDestroy(s->copy);
    if (s->d2h) cudaStreamDestroy(s->d2h);
    delete s->arena;
    delete s;
    return FIPT_OK;
}

// ---------------------------------------------------------------- check of the host order
extern "C" fipt_status fipt_debug_host_query_order(const fipt_query* q, int64_t n, const float* lo,
                                                   const float* hi, int32_t* order) {
    FIPT_REQUIRE(n >= 0 && n < ((int64_t)1 << 31), "bad point count");
    if (n == 0) return FIPT_OK;
    FIPT_REQUIRE(q && lo && hi && order, "NULL argument");
    host_query_order(q, n, lo, hi, order);
    return FIPT_OK;
}

// ---------------------------------------------------------------- check of the loop's bounded wait
extern "C" fipt_status fipt_debug_serve_wait_bound(int32_t wait_polls, int32_t* quit, int32_t* orphans,
                                                   int32_t* warps, double* seconds) {
    FIPT_REQUIRE(quit && orphans && warps && seconds, "NULL output");
    FIPT_REQUIRE(wait_polls >= 1 && wait_polls <= 65536, "wait_polls must be in [1, 65536]");
    const int n_warps = serve_loop_warps(1);
    ServeShared* sh = nullptr;
    ServeShared* sh_dev = nullptr;
    BakeChunk* chunks = nullptr;
    ServeCounters* ctr = nullptr;
    long long* orph = nullptr;
    int32_t* ints = nullptr;           // done count, done flag, status
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaHostAlloc(&sh, sizeof(ServeShared), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&sh_dev, sh, 0);
    if (e == cudaSuccess) e = cudaMalloc(&chunks, sizeof(BakeChunk));
    if (e == cudaSuccess) e = cudaMalloc(&ctr, sizeof(ServeCounters));
    if (e == cudaSuccess) e = cudaMalloc(&orph, sizeof(long long) * (size_t)n_warps);
    if (e == cudaSuccess) e = cudaMalloc(&ints, 3 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    fipt_status r = FIPT_OK;
    if (e == cudaSuccess) {
        std::memset(sh, 0, sizeof(ServeShared));
        e = cudaMemsetAsync(ctr, 0, sizeof(ServeCounters), st);      // nothing published, ever
        if (e == cudaSuccess) e = cudaMemsetAsync(ints, 0, 3 * sizeof(int32_t), st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess)
            r = launch_serve_bake(chunks, sh_dev, ctr, orph, orph, ints, ints + 1, ints + 2, wait_polls, 1, st, 0);
        if (e == cudaSuccess && r == FIPT_OK) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess && r == FIPT_OK) e = cudaStreamSynchronize(st);   // the launch ends by itself
        ServeCounters c{};
        if (e == cudaSuccess && r == FIPT_OK) e = cudaMemcpy(&c, ctr, sizeof(c), cudaMemcpyDeviceToHost);
        float ms = 0.0f;
        if (e == cudaSuccess && r == FIPT_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        *quit = c.quit;
        *orphans = c.n_out;
        *warps = n_warps;
        *seconds = 1e-3 * ms;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    cudaFree(ints);
    cudaFree(orph);
    cudaFree(ctr);
    cudaFree(chunks);
    if (sh) cudaFreeHost(sh);
    if (r != FIPT_OK) return r;
    return e == cudaSuccess ? FIPT_OK : fipt_check_cuda(e, "serve wait-bound check");
}
