// Emitter extraction (Sec. 4.4, Eq. 12).
//
// 1. Sample n locations uniformly on every triangle (square-root map of two
//    Philox uniforms, counter (t, j, 0x400, request)); the caller evaluates
//    its emission-mask field alpha there.
// 2. A triangle is an emitter when the mean of its n alphas exceeds the
//    threshold (0.01 in the paper); the mean is summed in sample order in
//    FP64, so the decision is deterministic.
// 3. With zero reflectance at emitters, the L1 problem of Eq. 12 is solved
//    per channel by the median of the radiance of the input pixels whose
//    first hit is the triangle.  The pixels that hit an emitter are first
//    gathered (in any order), sorted by triangle with the gathered count
//    read on the device, and each triangle's segment gives its count c;
//    the lower median (rank (c - 1) / 2 in each channel's order) is found
//    by radix selection on order-preserving bits of the values, which picks
//    the element a sort would put at that rank whatever the pixel order.
#include "fipt_internal.cuh"
#include "exact_sum.cuh"

namespace {

constexpr uint32_t EMIT_LANE = 0x400u;

// IDX: uint32_t when T * n < 2^32 (a 32-bit division splits the sample
// index), int64_t otherwise.  A block stages its PTS_THREADS points in
// shared memory and writes them as float4 (the block's 12 * PTS_THREADS
// bytes start 16-byte aligned when x is).
constexpr int PTS_THREADS = 256;

template <class IDX>
__global__ void __launch_bounds__(PTS_THREADS)
k_emit_points(const float4* __restrict__ tris, const int32_t* __restrict__ inv, int64_t T, int n, uint2 key,
              uint32_t rid, float* __restrict__ x) {
    __shared__ float4 buf[3 * PTS_THREADS / 4];
    float* sb = reinterpret_cast<float*>(buf);
    const int64_t total = T * n;
    const int64_t base = (int64_t)blockIdx.x * PTS_THREADS;
    const int64_t i = base + threadIdx.x;
    if (i < total) {
        const IDX t = (IDX)i / (IDX)n;
        const uint32_t j = (uint32_t)((IDX)i - t * (IDX)n);
        const int leaf = inv[t];
        const float4 p0 = __ldg(tris + 3 * leaf), p1 = __ldg(tris + 3 * leaf + 1), p2 = __ldg(tris + 3 * leaf + 2);
        const uint4 w = philox4x32_10(make_uint4((uint32_t)t, j, EMIT_LANE, rid), key);
        const float u1 = u24f(w.x), u2 = u24f(w.y);
        const float r1 = sqrtf(u1);
        const float b0 = 1.0f - r1, b1 = r1 * (1.0f - u2), b2 = r1 * u2;
        sb[3 * threadIdx.x + 0] = b0 * p0.x + b1 * p1.x + b2 * p2.x;
        sb[3 * threadIdx.x + 1] = b0 * p0.y + b1 * p1.y + b2 * p2.y;
        sb[3 * threadIdx.x + 2] = b0 * p0.z + b1 * p1.z + b2 * p2.z;
    }
    __syncthreads();
    const int64_t here = total - base < PTS_THREADS ? total - base : PTS_THREADS;
    if (here == PTS_THREADS && (reinterpret_cast<uintptr_t>(x) & 15) == 0) {
        float4* dst = reinterpret_cast<float4*>(x + 3 * base);
        if (threadIdx.x < 3 * PTS_THREADS / 4) dst[threadIdx.x] = buf[threadIdx.x];
    } else {
        for (int k = threadIdx.x; k < 3 * here; k += PTS_THREADS) x[3 * base + k] = sb[k];
    }
}

// A thread per triangle; its mean is the FP64 sum of its row of alpha in
// sample order over n.  Rows of up to CLS_STAGE_N samples are first copied
// to shared memory (a block's rows are contiguous: one coalesced float4
// stream).  A row within the exact range (exact_sum.cuh) is summed in
// integers in two passes (exponent range, then the sum), each thread
// starting at a column skewed by its index so that a warp's lanes read
// distinct banks (integer addition is associative, so the order does not
// change the sum); other rows (a wider exponent range, subnormals,
// infinities, NaNs) are summed in sample order in FP64.  The FP64 work
// left is one division per triangle, shared by the lanes of a warp.
constexpr int CLS_THREADS = 96;
constexpr int CLS_STAGE_N = 127;          // 96 rows x 127 floats = 48,768 B

template <bool STAGED>
__global__ void __launch_bounds__(CLS_THREADS)
k_emit_classify(const float* __restrict__ alpha, int64_t T, int n, double thr,
                double* __restrict__ mean, uint8_t* __restrict__ flag) {
    __shared__ float4 tile4[STAGED ? (CLS_THREADS * CLS_STAGE_N + 3) / 4 : 1];
    float* tile = reinterpret_cast<float*>(tile4);
    const int64_t t0 = (int64_t)blockIdx.x * CLS_THREADS;
    const int64_t t = t0 + threadIdx.x;
    const float* row;
    int c0 = 0;
    if (STAGED) {
        const int rows = (int)(T - t0 < CLS_THREADS ? T - t0 : CLS_THREADS);
        const float* src = alpha + t0 * (int64_t)n;
        const int cnt = rows * n;
        int done = 0;
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const int c4 = cnt >> 2;
            const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll 8
            for (int k = threadIdx.x; k < c4; k += CLS_THREADS) tile4[k] = __ldg(s4 + k);
            done = 4 * c4;
        }
#pragma unroll 4
        for (int k = done + threadIdx.x; k < cnt; k += CLS_THREADS) tile[k] = __ldg(src + k);
        __syncthreads();
        row = tile + threadIdx.x * n;
        c0 = threadIdx.x % n;
    } else {
        row = alpha + t * (int64_t)n;
    }
    if (t >= T) return;
    fipt_exact::Range rg;
    int c = c0;
    for (int j = 0; j < n; ++j) {
        rg.note(row[c]);
        c = c + 1 == n ? 0 : c + 1;
    }
    double s = 0.0;
    if (!rg.special() && rg.exact_for(n)) {
        const int emin = rg.emin();
        long long acc = 0;
        c = c0;
        for (int j = 0; j < n; ++j) {
            acc += fipt_exact::term(row[c], emin);
            c = c + 1 == n ? 0 : c + 1;
        }
        s = fipt_exact::scaled_double(acc, emin);
    } else {
        for (int j = 0; j < n; ++j) s += (double)row[j];
    }
    const double m = s / (double)n;
    if (mean) mean[t] = m;
    flag[t] = m > thr ? 1 : 0;
}

// Order-preserving map of float bits to unsigned (negative values flipped).
__device__ __forceinline__ uint32_t fkey(float v) {
    const uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float funkey(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// Gathers the pixels whose triangle is an emitter (one atomic per warp).
__global__ void k_emit_gather(const int32_t* __restrict__ tri, int64_t stride, int64_t P,
                              const uint8_t* __restrict__ flag, int64_t T, uint32_t* __restrict__ idx,
                              uint32_t* __restrict__ cnt) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool e = false;
    if (p < P) {
        const int32_t t = tri[p * stride];
        e = t >= 0 && t < T && flag[t];
    }
    const unsigned m = __ballot_sync(0xffffffffu, e);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (e) idx[base + __popc(m & ((1u << lane) - 1u))] = (uint32_t)p;
}

// Sort keys of the gathered pixels: their triangle (stable sort keeps
// gather order within a triangle, which the median does not depend on).
__global__ void k_emit_tri_keys(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ cnt,
                                const int32_t* __restrict__ tri, int64_t stride, uint32_t* __restrict__ keys,
                                uint32_t* __restrict__ vals) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= (int64_t)*cnt) return;
    const int64_t p = idx[j];
    keys[j] = (uint32_t)tri[p * stride];
    vals[j] = (uint32_t)p;
}

// Segment bounds of every triangle with pixels, and the list of those
// triangles (one atomic per warp; the list's order does not matter).
__global__ void k_emit_bounds(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ cnt, int64_t T,
                              int32_t* __restrict__ start, int32_t* __restrict__ end, uint32_t* __restrict__ segs,
                              uint32_t* __restrict__ nseg) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t P = *cnt;
    const int lane = threadIdx.x & 31;
    bool first = false;
    uint32_t s = 0;
    if (j < P) {
        s = keys[j];
        if (s < (uint64_t)T) {
            first = j == 0 || keys[j - 1] != s;
            if (first) start[s] = (int32_t)j;
            if (j == P - 1 || keys[j + 1] != s) end[s] = (int32_t)j;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, first);
    if (m == 0) return;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(nseg, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (first) segs[base + __popc(m & ((1u << lane) - 1u))] = s;
}

// The three channels' order-preserving keys of the sorted pixels, laid out
// [channel][sorted position] so that a triangle's keys are contiguous.
__global__ void k_emit_chan_keys(const uint32_t* __restrict__ pix, const uint32_t* __restrict__ cnt,
                                 const float* __restrict__ rgb, int64_t P, uint32_t* __restrict__ keys3) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= (int64_t)*cnt) return;
    const int64_t p = pix[j];
#pragma unroll
    for (int c = 0; c < 3; ++c) keys3[c * P + j] = fkey(rgb[3 * p + c]);
}

constexpr int SEL_THREADS = 256;            // a block per triangle

// Lower median of each channel of triangle t's pixels (positions a..e of
// keys3) by radix selection on the order-preserving keys: four 8-bit
// digits from the top, each pass counting the candidates' digit in a
// shared histogram and keeping the bucket that holds rank (n - 1) / 2.  The
// selected key is the one a sort would put at that rank, so the result
// equals the sorted lower median.  Triangles without pixels get 0 and
// count 0 (set beforehand).  Persistent: the blocks take the listed
// triangles in turn.
__global__ void __launch_bounds__(SEL_THREADS)
k_emit_select(const uint32_t* __restrict__ keys3, int64_t P, const int32_t* __restrict__ start,
              const int32_t* __restrict__ end, const uint32_t* __restrict__ segs, const uint32_t* __restrict__ nseg,
              float* __restrict__ Le, int32_t* __restrict__ count) {
    __shared__ uint32_t hist[256];
    __shared__ uint32_t pick[2];
    const int tid = threadIdx.x;
    const uint32_t ns = *nseg;
    for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
        const int64_t t = segs[si];
        const int32_t a = start[t];                         // the same for the whole block
        const int32_t n = end[t] - a + 1;
        for (int c = 0; c < 3; ++c) {
            const uint32_t* key = keys3 + c * P + a;
            uint32_t prefix = 0, mask = 0, k = (uint32_t)(n - 1) / 2;
            for (int shift = 24; shift >= 0; shift -= 8) {
                hist[tid] = 0;
                __syncthreads();
                for (int32_t j = tid; j < n; j += SEL_THREADS) {
                    const uint32_t v = key[j];
                    if ((v & mask) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (tid < 32) {                             // warp 0 finds the bucket holding rank k
                    uint32_t h[8], sum = 0;
    #pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        h[b] = hist[tid * 8 + b];
                        sum += h[b];
                    }
                    uint32_t incl = sum;
    #pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (tid >= o) incl += y;
                    }
                    const uint32_t excl = incl - sum;
                    if (excl <= k && k < incl) {
                        uint32_t run = excl;
                        for (int b = 0; b < 8; ++b) {
                            if (k < run + h[b]) {
                                pick[0] = (uint32_t)(tid * 8 + b);
                                pick[1] = run;
                                break;
                            }
                            run += h[b];
                        }
                    }
                }
                __syncthreads();
                k -= pick[1];
                prefix |= pick[0] << shift;
                mask |= 255u << shift;
                __syncthreads();                            // pick[] and hist[] are reused
            }
            if (tid == 0) Le[3 * t + c] = funkey(prefix);
        }
        if (count && tid == 0) count[t] = n;
    }
}

__global__ void k_set_emission(const float* __restrict__ Le, const int32_t* __restrict__ order,
                               int64_t T, float4* __restrict__ shade) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    const int64_t t = order[leaf];
    shade[2 * leaf] = make_float4(Le[3 * t], Le[3 * t + 1], Le[3 * t + 2], 0.0f);
}

struct EmitLayout {
    uint32_t *keys, *keys_alt, *vals, *vals_alt, *hist, *idx, *keys3, *segs, *cnt;
    int32_t *start, *end;
    size_t bytes;
};

EmitLayout carve(void* ws, int64_t P, int64_t T) {
    Carver c{static_cast<char*>(ws), 0};
    EmitLayout L;
    const int64_t p1 = P > 0 ? P : 1, t1 = T > 0 ? T : 1;
    L.keys = c.take<uint32_t>((size_t)p1);
    L.keys_alt = c.take<uint32_t>((size_t)p1);
    L.vals = c.take<uint32_t>((size_t)p1);
    L.vals_alt = c.take<uint32_t>((size_t)p1);
    L.hist = c.take<uint32_t>(radix_sort_scratch_bytes(p1) / sizeof(uint32_t));
    L.start = c.take<int32_t>((size_t)t1);
    L.end = c.take<int32_t>((size_t)t1);
    L.idx = c.take<uint32_t>((size_t)p1);
    L.keys3 = c.take<uint32_t>((size_t)(3 * p1));
    L.segs = c.take<uint32_t>((size_t)t1);
    L.cnt = c.take<uint32_t>(2);                       // gathered pixels, listed triangles
    L.bytes = c.off + 256;
    return L;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" fipt_status fipt_emitter_sample_points(fipt_scene* s, uint64_t seed, uint32_t request_id,
                                                  int32_t n_per_tri, float* x, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(n_per_tri >= 1 && n_per_tri <= (1 << 20), "n_per_tri must be in [1, 2^20]");
    FIPT_REQUIRE(s->T * (int64_t)n_per_tri < ((int64_t)1 << 39), "T * n_per_tri must be < 2^39");
    if (s->T == 0) return FIPT_OK;
    FIPT_REQUIRE(x && fipt_aligned(x, 4), "x is NULL or misaligned");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    const int64_t n = s->T * n_per_tri;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if (n < ((int64_t)1 << 32))
        FIPT_LAUNCH(k_emit_points<uint32_t>, blocks(n, PTS_THREADS), PTS_THREADS, 0,
                    static_cast<cudaStream_t>(stream), s->tris, s->inv, s->T, n_per_tri, key, request_id, x);
    else
        FIPT_LAUNCH(k_emit_points<int64_t>, blocks(n, PTS_THREADS), PTS_THREADS, 0,
                    static_cast<cudaStream_t>(stream), s->tris, s->inv, s->T, n_per_tri, key, request_id, x);
    FIPT_LAUNCHED("emitter sample points");
    return FIPT_OK;
}

extern "C" fipt_status fipt_emitter_classify(const float* alpha, int64_t T, int32_t n_per_tri,
                                             float threshold, double* mean_alpha, uint8_t* is_emitter,
                                             fipt_stream stream) {
    FIPT_REQUIRE(T >= 0 && T < ((int64_t)1 << 31), "bad T");
    FIPT_REQUIRE(n_per_tri >= 1 && n_per_tri <= (1 << 20), "n_per_tri must be in [1, 2^20]");
    if (T == 0) return FIPT_OK;
    FIPT_REQUIRE(alpha && is_emitter && fipt_aligned(alpha, 4), "alpha / is_emitter NULL or misaligned");
    FIPT_REQUIRE(!mean_alpha || fipt_aligned(mean_alpha, 8), "mean_alpha misaligned");
    const unsigned nb = blocks(T, CLS_THREADS);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_per_tri <= CLS_STAGE_N)
        FIPT_LAUNCH(k_emit_classify<true>, nb, CLS_THREADS, 0, st, alpha, T, n_per_tri, (double)threshold,
                    mean_alpha, is_emitter);
    else
        FIPT_LAUNCH(k_emit_classify<false>, nb, CLS_THREADS, 0, st, alpha, T, n_per_tri, (double)threshold,
                    mean_alpha, is_emitter);
    FIPT_LAUNCHED("emitter classify");
    return FIPT_OK;
}

extern "C" fipt_status fipt_emitter_radiance_workspace_size(int64_t P, int64_t T, size_t* bytes) {
    FIPT_REQUIRE(bytes && P >= 0 && P < ((int64_t)1 << 31) && T >= 0 && T < ((int64_t)1 << 31),
                 "bad arguments");
    *bytes = carve(nullptr, P, T).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_emitter_radiance(const int32_t* tri, int64_t tri_stride, const float* rgb,
                                             int64_t P, const uint8_t* is_emitter, int64_t T, float* Le,
                                             int32_t* count, void* ws, size_t ws_bytes,
                                             fipt_stream stream) {
    FIPT_REQUIRE(P >= 0 && P < ((int64_t)1 << 31) && T >= 0 && T < ((int64_t)1 << 31) && tri_stride >= 1,
                 "bad sizes");
    if (T == 0) return FIPT_OK;
    FIPT_REQUIRE(is_emitter && Le && fipt_aligned(Le, 4), "is_emitter / Le NULL or misaligned");
    FIPT_REQUIRE(!count || fipt_aligned(count, 4), "count misaligned");
    FIPT_REQUIRE(P == 0 || (tri && rgb && fipt_aligned(tri, 4) && fipt_aligned(rgb, 4)),
                 "tri / rgb NULL or misaligned");
    EmitLayout Y = carve(ws, P, T);
    if (!ws || ws_bytes < Y.bytes || !fipt_aligned(ws, 256))
        return fipt_set_error(FIPT_ERR_WORKSPACE, "emitter workspace %zu < %zu bytes (256-aligned)",
                              ws_bytes, Y.bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FIPT_CUDA(cudaMemsetAsync(Y.start, 0xFF, sizeof(int32_t) * (size_t)T, st));
    FIPT_CUDA(cudaMemsetAsync(Y.end, 0xFF, sizeof(int32_t) * (size_t)T, st));
    int bits = 0;
    while (((int64_t)1 << bits) < T) ++bits;               // triangle ids 0..T-1
    bits = bits > 0 ? (bits + 7) & ~7 : 8;
    FIPT_CUDA(cudaMemsetAsync(Y.cnt, 0, 2 * sizeof(uint32_t), st));
    FIPT_CUDA(cudaMemsetAsync(Le, 0, 3 * sizeof(float) * (size_t)T, st));
    if (count) FIPT_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)T, st));
    uint32_t* sv = Y.vals;
    if (P > 0) {
        FIPT_LAUNCH(k_emit_gather, blocks(P, 256), 256, 0, st, tri, tri_stride, P, is_emitter, T, Y.idx, Y.cnt);
        FIPT_LAUNCH(k_emit_tri_keys, blocks(P, 256), 256, 0, st, Y.idx, Y.cnt, tri, tri_stride, Y.keys, Y.vals);
        uint32_t* sk;
        fipt_status r = radix_sort_pairs<uint32_t>(Y.keys, Y.keys_alt, Y.vals, Y.vals_alt, Y.hist, P, bits, st,
                                                   &sk, &sv, Y.cnt);
        if (r != FIPT_OK) return r;
        FIPT_LAUNCH(k_emit_bounds, blocks(P, 256), 256, 0, st, sk, Y.cnt, T, Y.start, Y.end, Y.segs, Y.cnt + 1);
        FIPT_LAUNCH(k_emit_chan_keys, blocks(P, 256), 256, 0, st, sv, Y.cnt, rgb, P, Y.keys3);
        int dev = 0, sms = 0;
        FIPT_CUDA(cudaGetDevice(&dev));
        FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FIPT_LAUNCH(k_emit_select, (unsigned)(8 * sms), SEL_THREADS, 0, st, Y.keys3, P, Y.start, Y.end, Y.segs,
                    Y.cnt + 1, Le, count);
    }
    FIPT_LAUNCHED("emitter radiance");
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_set_emission(fipt_scene* s, const float* Le, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(s->T == 0 || (Le && fipt_aligned(Le, 4)), "Le is NULL or misaligned");
    if (s->T == 0) return FIPT_OK;
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FIPT_LAUNCH(k_set_emission, blocks(s->T, 256), 256, 0, st, Le, s->order, s->T, s->shade);
    return rebuild_emitter_table(s, st);
}
