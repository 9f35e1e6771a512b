// Emitter extraction (Sec. 4.4, Eq. 12).
//
// 1. Sample n locations uniformly on every triangle (square-root map of two
//    Philox uniforms, counter (t, j, 0x400, request)); the caller evaluates
//    its emission-mask field alpha there.
// 2. A triangle is an emitter when the mean of its n alphas exceeds the
//    threshold (0.01 in the paper); the mean is the FP64 sum in sample
//    order over n (reached by exact integer sums where those apply), so
//    the decision is deterministic.
// 3. With zero reflectance at emitters, the L1 problem of Eq. 12 is solved
//    per channel by the median of the radiance of the input pixels whose
//    first hit is the triangle.  The pixels on emitter triangles are
//    grouped by triangle with a counting sort: per-triangle counts, a scan
//    over the triangles for each one's segment, and a scatter of each
//    pixel's three channel keys into its segment (in any order within it);
//    the lower median (rank (c - 1) / 2 of a segment's c keys in each
//    channel's order) is found on order-preserving bits of the values, by
//    ranking for segments of at most 32 keys and by radix selection for
//    longer ones; both pick the element a sort would put at that rank
//    whatever the order within the segment.
#include "fipt_internal.cuh"
#include "exact_sum.cuh"

namespace {

constexpr uint32_t EMIT_LANE = 0x400u;

// Division of 32-bit indices by the invariant n (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with
// l = ceil(log2 n) and m = floor(2^32 (2^l - n) / n) + 1, every 32-bit i
// has i / n = (t + ((i - t) >> min(l, 1))) >> max(l - 1, 0), t = mulhi(m, i).
struct DivN {
    uint32_t m;
    int s1, s2;
};

DivN div_by(uint32_t n) {
    int l = 0;
    while (((uint64_t)1 << l) < n) ++l;
    const uint64_t m = (((uint64_t)1 << 32) * (((uint64_t)1 << l) - n)) / n + 1;
    return DivN{(uint32_t)m, l < 1 ? l : 1, l > 1 ? l - 1 : 0};
}

// i / n for the divisor d was made for (device: one multiply-high).
__host__ __device__ __forceinline__ uint32_t div_apply(const DivN& d, uint32_t i) {
#ifdef __CUDA_ARCH__
    const uint32_t hi = __umulhi(d.m, i);
#else
    const uint32_t hi = (uint32_t)(((uint64_t)d.m * i) >> 32);
#endif
    return (hi + ((i - hi) >> d.s1)) >> d.s2;
}

__global__ void k_debug_divide(DivN d, const uint32_t* __restrict__ i, int64_t count,
                               uint32_t* __restrict__ out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < count) out[k] = div_apply(d, i[k]);
}

// IDX: uint32_t when T * n < 2^32 (the sample index splits by the
// multiply-high division above), int64_t otherwise.  A block stages its
// PTS_THREADS points in shared memory and writes them as float4 (the
// block's 12 * PTS_THREADS bytes start 16-byte aligned when x is).
constexpr int PTS_THREADS = 256;

template <class IDX>
__global__ void __launch_bounds__(PTS_THREADS)
k_emit_points(const float4* __restrict__ tris, const int32_t* __restrict__ inv, int64_t T, int n, DivN dn,
              uint2 key, uint32_t rid, float* __restrict__ x) {
    __shared__ float4 buf[3 * PTS_THREADS / 4];
    float* sb = reinterpret_cast<float*>(buf);
    const int64_t total = T * n;
    const int64_t base = (int64_t)blockIdx.x * PTS_THREADS;
    const int64_t i = base + threadIdx.x;
    if (i < total) {
        IDX t;
        if constexpr (sizeof(IDX) == 4) {
            t = div_apply(dn, (uint32_t)i);
        } else {
            t = (IDX)i / (IDX)n;
        }
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

// Pixel p's triangle when it is an emitter, else -1.
__device__ __forceinline__ int32_t emitter_of(const int32_t* __restrict__ tri, int64_t stride, int64_t p,
                                              const uint8_t* __restrict__ flag, int64_t T) {
    const int32_t t = tri[p * stride];
    return (t >= 0 && t < T && flag[t]) ? t : -1;
}

// Pixels per emitter triangle: the lanes of a warp on the same triangle
// (grouped by __match_any_sync) add with one atomic.
__global__ void k_emit_count(const int32_t* __restrict__ tri, int64_t stride, int64_t P,
                             const uint8_t* __restrict__ flag, int64_t T, uint32_t* __restrict__ tcount) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t t = p < P ? emitter_of(tri, stride, p, flag, T) : -1;
    const unsigned act = __ballot_sync(0xffffffffu, t >= 0);
    if (t < 0) return;
    const unsigned same = __match_any_sync(act, (unsigned)t);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&tcount[t], (uint32_t)__popc(same));
}

// Segments of the triangles (tiles of SEG_TILE triangles): k_emit_seg_tiles
// sums each tile's pixel counts and counts its triangles with pixels,
// k_emit_seg_scan turns both into offsets (one block; cnt[0] = pixels on
// emitters, cnt[1] = triangles with pixels), k_emit_seg_apply gives each
// triangle with pixels its segment [start, end], a cursor at start, and its
// place in the list of such triangles (in triangle order).
constexpr int SEG_TILE = 1024;

// Exclusive prefix of v over a block of SEG_TILE threads; total receives
// the block's sum.  ws: 33 words of shared memory.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t v, uint32_t* ws, uint32_t& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        const uint32_t s0 = ws[lane];
        uint32_t s = s0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s - s0;
        if (lane == 31) ws[32] = s;
    }
    __syncthreads();
    const uint32_t r = ws[w] + x - v;
    total = ws[32];
    __syncthreads();                                       // ws is reused by the next call
    return r;
}

__global__ void __launch_bounds__(SEG_TILE)
k_emit_seg_tiles(const uint32_t* __restrict__ tcount, int64_t T, uint32_t* __restrict__ tsum,
                 uint32_t* __restrict__ tnz) {
    __shared__ uint32_t ws[33];
    const int64_t t = blockIdx.x * (int64_t)SEG_TILE + threadIdx.x;
    const uint32_t c = t < T ? tcount[t] : 0u;
    uint32_t s, z;
    block_exclusive(c, ws, s);
    block_exclusive(c > 0u ? 1u : 0u, ws, z);
    if (threadIdx.x == 0) {
        tsum[blockIdx.x] = s;
        tnz[blockIdx.x] = z;
    }
}

__global__ void __launch_bounds__(SEG_TILE)
k_emit_seg_scan(uint32_t* __restrict__ tsum, uint32_t* __restrict__ tnz, int64_t nt, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t ws[33];
    uint32_t carry_s = 0, carry_z = 0;
    for (int64_t base = 0; base < nt; base += SEG_TILE) {
        const int64_t i = base + threadIdx.x;
        uint32_t ts, tz;
        const uint32_t es = block_exclusive(i < nt ? tsum[i] : 0u, ws, ts);
        const uint32_t ez = block_exclusive(i < nt ? tnz[i] : 0u, ws, tz);
        if (i < nt) {
            tsum[i] = carry_s + es;
            tnz[i] = carry_z + ez;
        }
        carry_s += ts;
        carry_z += tz;
    }
    if (threadIdx.x == 0) {
        cnt[0] = carry_s;
        cnt[1] = carry_z;
    }
}

__global__ void __launch_bounds__(SEG_TILE)
k_emit_seg_apply(const uint32_t* __restrict__ tcount, int64_t T, const uint32_t* __restrict__ tsum,
                 const uint32_t* __restrict__ tnz, int32_t* __restrict__ start, int32_t* __restrict__ end,
                 uint32_t* __restrict__ cursor, uint32_t* __restrict__ segs) {
    __shared__ uint32_t ws[33];
    const int64_t t = blockIdx.x * (int64_t)SEG_TILE + threadIdx.x;
    const uint32_t c = t < T ? tcount[t] : 0u;
    uint32_t total;
    const uint32_t ps = tsum[blockIdx.x] + block_exclusive(c, ws, total);
    const uint32_t pz = tnz[blockIdx.x] + block_exclusive(c > 0u ? 1u : 0u, ws, total);
    if (c > 0u) {
        start[t] = (int32_t)ps;
        end[t] = (int32_t)(ps + c - 1u);
        cursor[t] = ps;
        segs[pz] = (uint32_t)t;
    }
}

// Each emitter pixel's three channel keys go to its triangle's segment,
// laid out [channel][position] (P positions per channel); the lanes of a
// warp on the same triangle take consecutive positions with one atomic.
__global__ void k_emit_scatter(const int32_t* __restrict__ tri, int64_t stride, int64_t P,
                               const uint8_t* __restrict__ flag, int64_t T, const float* __restrict__ rgb,
                               uint32_t* __restrict__ cursor, uint32_t* __restrict__ keys3) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t t = p < P ? emitter_of(tri, stride, p, flag, T) : -1;
    const unsigned act = __ballot_sync(0xffffffffu, t >= 0);
    if (t < 0) return;
    const int lane = threadIdx.x & 31;
    const unsigned same = __match_any_sync(act, (unsigned)t);
    const int leader = __ffs(same) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&cursor[t], (uint32_t)__popc(same));
    base = __shfl_sync(act, base, leader);
    const int64_t pos = base + __popc(same & ((1u << lane) - 1u));
#pragma unroll
    for (int c = 0; c < 3; ++c) keys3[c * P + pos] = fkey(rgb[3 * p + c]);
}

// Lower median of each channel of the triangles with at most 32 pixels, a
// warp per triangle: lane j holds the triangle's j-th key, counts the keys
// ordered before it by (key, position) with n shuffles, and the lane whose
// count is (n - 1) / 2 holds the key a sort would put at that rank.
// Triangles with more pixels are left to k_emit_select.
constexpr int SEL_SMALL = 32;

__global__ void k_emit_select_small(const uint32_t* __restrict__ keys3, int64_t P, const int32_t* __restrict__ start,
                                    const int32_t* __restrict__ end, const uint32_t* __restrict__ segs,
                                    const uint32_t* __restrict__ nseg, float* __restrict__ Le,
                                    int32_t* __restrict__ count) {
    const int lane = threadIdx.x & 31;
    const uint32_t ns = *nseg;
    const uint32_t nwarps = gridDim.x * (blockDim.x / 32);
    for (uint32_t si = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); si < ns; si += nwarps) {
        const int64_t t = segs[si];
        const int32_t a = start[t];
        const int32_t n = end[t] - a + 1;
        if (n > SEL_SMALL) continue;                      // whole warp
        const int k = (n - 1) / 2;
        for (int c = 0; c < 3; ++c) {
            const uint32_t mine = lane < n ? keys3[c * P + a + lane] : 0xFFFFFFFFu;
            int before = 0;
            for (int j = 0; j < n; ++j) {
                const uint32_t v = __shfl_sync(0xffffffffu, mine, j);
                before += (v < mine || (v == mine && j < lane)) ? 1 : 0;
            }
            if (lane < n && before == k) Le[3 * t + c] = funkey(mine);
        }
        if (count && lane == 0) count[t] = n;
    }
}

constexpr int SEL_THREADS = 256;            // a block per triangle

// Lower median of each channel of triangle t's pixels (positions a..e of
// keys3) by radix selection on the order-preserving keys: four 8-bit
// digits from the top, each pass counting the candidates' digit in a
// shared histogram and keeping the bucket that holds rank (n - 1) / 2; the
// three channels are selected in the same passes (three histograms, a warp
// each to find the bucket).  The selected key is the one a sort would put
// at that rank, so the result equals the sorted lower median.  Triangles
// without pixels get 0 and count 0 (set beforehand).  Persistent: the
// blocks take the listed triangles with more than SEL_SMALL pixels in turn.
__global__ void __launch_bounds__(SEL_THREADS)
k_emit_select(const uint32_t* __restrict__ keys3, int64_t P, const int32_t* __restrict__ start,
              const int32_t* __restrict__ end, const uint32_t* __restrict__ segs, const uint32_t* __restrict__ nseg,
              float* __restrict__ Le, int32_t* __restrict__ count) {
    __shared__ uint32_t hist[3][256];
    __shared__ uint32_t pick[3][2];
    const int tid = threadIdx.x;
    const uint32_t ns = *nseg;
    for (uint32_t si = blockIdx.x; si < ns; si += gridDim.x) {
        const int64_t t = segs[si];
        const int32_t a = start[t];                         // the same for the whole block
        const int32_t n = end[t] - a + 1;
        if (n <= SEL_SMALL) continue;                       // taken by k_emit_select_small
        const uint32_t* key0 = keys3 + a;
        uint32_t prefix[3] = {0u, 0u, 0u}, kk[3];
        kk[0] = kk[1] = kk[2] = (uint32_t)(n - 1) / 2;
        uint32_t mask = 0;
        for (int shift = 24; shift >= 0; shift -= 8) {
            for (int i = tid; i < 3 * 256; i += SEL_THREADS) (&hist[0][0])[i] = 0;
            __syncthreads();
            for (int32_t j = tid; j < n; j += SEL_THREADS) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const uint32_t v = key0[c * P + j];
                    if ((v & mask) == prefix[c]) atomicAdd(&hist[c][(v >> shift) & 255u], 1u);
                }
            }
            __syncthreads();
            if (tid < 96) {                                 // warp c finds channel c's bucket holding rank kk[c]
                const int c = tid >> 5, lane = tid & 31;
                const uint32_t k = c == 0 ? kk[0] : (c == 1 ? kk[1] : kk[2]);
                uint32_t h[8], sum = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    h[b] = hist[c][lane * 8 + b];
                    sum += h[b];
                }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const uint32_t excl = incl - sum;
                if (excl <= k && k < incl) {
                    uint32_t run = excl;
                    for (int b = 0; b < 8; ++b) {
                        if (k < run + h[b]) {
                            pick[c][0] = (uint32_t)(lane * 8 + b);
                            pick[c][1] = run;
                            break;
                        }
                        run += h[b];
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                kk[c] -= pick[c][1];
                prefix[c] |= pick[c][0] << shift;
            }
            mask |= 255u << shift;
            __syncthreads();                                // pick[] and hist[] are reused
        }
        if (tid < 3) Le[3 * t + tid] = funkey(tid == 0 ? prefix[0] : (tid == 1 ? prefix[1] : prefix[2]));
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
    uint32_t *tcount, *cursor, *segs, *tsum, *tnz, *keys3, *cnt;
    int32_t *start, *end;
    size_t bytes;
};

EmitLayout carve(void* ws, int64_t P, int64_t T) {
    Carver c{static_cast<char*>(ws), 0};
    EmitLayout L;
    const int64_t p1 = P > 0 ? P : 1, t1 = T > 0 ? T : 1;
    L.tcount = c.take<uint32_t>((size_t)t1);
    L.cursor = c.take<uint32_t>((size_t)t1);
    L.start = c.take<int32_t>((size_t)t1);
    L.end = c.take<int32_t>((size_t)t1);
    L.segs = c.take<uint32_t>((size_t)t1);
    L.tsum = c.take<uint32_t>((size_t)((t1 + SEG_TILE - 1) / SEG_TILE));
    L.tnz = c.take<uint32_t>((size_t)((t1 + SEG_TILE - 1) / SEG_TILE));
    L.keys3 = c.take<uint32_t>((size_t)(3 * p1));
    L.cnt = c.take<uint32_t>(2);                       // pixels on emitters, triangles with pixels
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
    const DivN dn = div_by((uint32_t)n_per_tri);
    if (n < ((int64_t)1 << 32))
        FIPT_LAUNCH(k_emit_points<uint32_t>, blocks(n, PTS_THREADS), PTS_THREADS, 0,
                    static_cast<cudaStream_t>(stream), s->tris, s->inv, s->T, n_per_tri, dn, key, request_id, x);
    else
        FIPT_LAUNCH(k_emit_points<int64_t>, blocks(n, PTS_THREADS), PTS_THREADS, 0,
                    static_cast<cudaStream_t>(stream), s->tris, s->inv, s->T, n_per_tri, dn, key, request_id, x);
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
    FIPT_CUDA(cudaMemsetAsync(Le, 0, 3 * sizeof(float) * (size_t)T, st));
    if (count) FIPT_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)T, st));
    if (P > 0) {
        FIPT_CUDA(cudaMemsetAsync(Y.tcount, 0, sizeof(uint32_t) * (size_t)T, st));
        FIPT_LAUNCH(k_emit_count, blocks(P, 256), 256, 0, st, tri, tri_stride, P, is_emitter, T, Y.tcount);
        const int64_t nt = (T + SEG_TILE - 1) / SEG_TILE;
        FIPT_LAUNCH(k_emit_seg_tiles, (unsigned)nt, SEG_TILE, 0, st, Y.tcount, T, Y.tsum, Y.tnz);
        FIPT_LAUNCH(k_emit_seg_scan, 1, SEG_TILE, 0, st, Y.tsum, Y.tnz, nt, Y.cnt);
        FIPT_LAUNCH(k_emit_seg_apply, (unsigned)nt, SEG_TILE, 0, st, Y.tcount, T, Y.tsum, Y.tnz, Y.start, Y.end,
                    Y.cursor, Y.segs);
        FIPT_LAUNCH(k_emit_scatter, blocks(P, 256), 256, 0, st, tri, tri_stride, P, is_emitter, T, rgb, Y.cursor,
                    Y.keys3);
        int dev = 0, sms = 0;
        FIPT_CUDA(cudaGetDevice(&dev));
        FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FIPT_LAUNCH(k_emit_select_small, (unsigned)(8 * sms), 256, 0, st, Y.keys3, P, Y.start, Y.end, Y.segs,
                    Y.cnt + 1, Le, count);
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

extern "C" fipt_status fipt_debug_divide(uint32_t n, const uint32_t* i, int64_t count, uint32_t* out,
                                         int32_t on_device, fipt_stream stream) {
    FIPT_REQUIRE(n >= 1 && count >= 0 && (count == 0 || (i && out)), "bad arguments");
    const DivN d = div_by(n);
    if (!on_device) {
        for (int64_t k = 0; k < count; ++k) out[k] = div_apply(d, i[k]);
        return FIPT_OK;
    }
    if (count == 0) return FIPT_OK;
    FIPT_LAUNCH(k_debug_divide, (unsigned)((count + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream),
                d, i, count, out);
    FIPT_LAUNCHED("debug_divide");
    return FIPT_OK;
}
