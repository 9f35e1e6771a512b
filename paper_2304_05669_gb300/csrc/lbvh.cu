// Scene build on the device: linear BVH (Karras 2012) over the triangles.
//
//   bounds  -> vertex bounding box (order-preserving int atomics, exact)
//   morton  -> 63-bit Morton code of each triangle's box centre, quantised
//              with individually rounded IEEE double operations
//   sort    -> stable LSD radix sort of (code, triangle index)
//   karras  -> binary radix tree over the sorted codes (ties by index)
//   pack    -> triangles and their radiance in sorted (leaf) order
//   refit   -> bottom-up node boxes with per-node arrival counters
#include "fipt_internal.cuh"

namespace {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int RADIX = 256;
constexpr int SCAN_THREADS = 1024;

int64_t sort_blocks(int64_t n) { return (n + SORT_TILE - 1) / SORT_TILE; }

// ---------------------------------------------------------------- radix sort
template <class K>
__global__ void __launch_bounds__(SORT_THREADS)
k_sort_hist(const K* __restrict__ keys, int64_t n, const uint32_t* __restrict__ n_dev, int shift,
            uint32_t* __restrict__ hist) {
    __shared__ uint32_t cnt[RADIX];
    cnt[threadIdx.x] = 0;
    if (n_dev && (int64_t)*n_dev < n) n = *n_dev;      // a device-side count bounds the keys
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
#pragma unroll
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int64_t i = base + it * SORT_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & (RADIX - 1)], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of m counters in one block (digit-major histogram).
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_single(uint32_t* __restrict__ a, int64_t m) {
    __shared__ uint32_t part[SCAN_THREADS];
    const int64_t per = (m + SCAN_THREADS - 1) / SCAN_THREADS;
    const int64_t beg = threadIdx.x * per;
    const int64_t end = beg + per < m ? beg + per : m;
    uint32_t s = 0;
    for (int64_t i = beg; i < end; ++i) s += a[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < SCAN_THREADS; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - s;
    for (int64_t i = beg; i < end; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
}

// Multi-block exclusive scan for large histograms: k_scan_reduce sums
// chunks of SCAN_CHUNK counters, k_scan_single scans those sums, and
// k_scan_apply scans each chunk from its scanned sum.  Thread i of a block
// owns counters 4i .. 4i+3 of the chunk.
constexpr int SCAN_CHUNK = 4 * SCAN_THREADS;

__device__ __forceinline__ uint4 load4(const uint32_t* a, int64_t i, int64_t m) {
    if (i + 3 < m) return *reinterpret_cast<const uint4*>(a + i);
    return make_uint4(i < m ? a[i] : 0u, i + 1 < m ? a[i + 1] : 0u, i + 2 < m ? a[i + 2] : 0u, 0u);
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_reduce(const uint32_t* __restrict__ a, int64_t m, uint32_t* __restrict__ bsum) {
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    const int64_t i = (int64_t)blockIdx.x * SCAN_CHUNK + 4 * threadIdx.x;
    const uint4 v = load4(a, i, m);
    uint32_t t = v.x + v.y + v.z + v.w;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t u = wsum[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = u;
    }
}

__global__ void __launch_bounds__(SCAN_THREADS)
k_scan_apply(uint32_t* __restrict__ a, int64_t m, const uint32_t* __restrict__ bsum) {
    __shared__ uint32_t wsum[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * SCAN_CHUNK + 4 * threadIdx.x;
    const uint4 v = load4(a, i, m);
    const uint32_t t = v.x + v.y + v.z + v.w;
    uint32_t incl = t;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t u = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        wsum[lane] = u;
    }
    __syncthreads();
    uint32_t run = bsum[blockIdx.x] + (warp > 0 ? wsum[warp - 1] : 0u) + incl - t;
    const uint32_t e0 = run, e1 = e0 + v.x, e2 = e1 + v.y, e3 = e2 + v.z;
    if (i + 3 < m) {
        *reinterpret_cast<uint4*>(a + i) = make_uint4(e0, e1, e2, e3);
    } else {
        if (i < m) a[i] = e0;
        if (i + 1 < m) a[i + 1] = e1;
        if (i + 2 < m) a[i + 2] = e2;
    }
}

// Stable scatter: an element's rank among equal digits in its tile follows
// (iteration, warp, lane), i.e. index order.
template <class K>
__global__ void __launch_bounds__(SORT_THREADS)
k_sort_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* __restrict__ kout,
               uint32_t* __restrict__ vout, int64_t n, const uint32_t* __restrict__ n_dev, int shift,
               const uint32_t* __restrict__ hist) {
    if (n_dev && (int64_t)*n_dev < n) n = *n_dev;
    if ((int64_t)blockIdx.x * SORT_TILE >= n) return;   // the whole tile is past the keys
    constexpr int WARPS = SORT_THREADS / 32;
    __shared__ uint32_t base_off[RADIX];
    __shared__ uint32_t run[RADIX];
    __shared__ uint32_t wcnt[WARPS][RADIX];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    base_off[tid] = hist[(int64_t)tid * gridDim.x + blockIdx.x];
    run[tid] = 0;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int it = 0; it < SORT_ITEMS; ++it) {
        const int64_t i = base + it * SORT_THREADS + tid;
        const bool valid = i < n;
        K k = 0;
        uint32_t v = 0;
        uint32_t digit = RADIX;
        if (valid) {
            k = kin[i];
            v = vin[i];
            digit = (uint32_t)(k >> shift) & (RADIX - 1);
        }
#pragma unroll
        for (int w = 0; w < WARPS; ++w) wcnt[w][tid] = 0;
        __syncthreads();
        const uint32_t peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t r = run[tid];
#pragma unroll
            for (int w = 0; w < WARPS; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = r;
                r += c;
            }
            run[tid] = r;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = base_off[digit] + wcnt[warp][digit] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- bounds
__global__ void k_bounds_init(SceneConst* c) {
    if (threadIdx.x == 0) {
        c->n_emit = 0;
        c->A_emit = 0.0;
    }
    if (threadIdx.x < 3) {
        c->lo_key[threadIdx.x] = float_to_ordered(__int_as_float(0x7f800000));   // +inf
        c->hi_key[threadIdx.x] = float_to_ordered(__int_as_float(0xff800000));   // -inf
    }
}

__global__ void k_bounds(const float* __restrict__ V, int64_t nV, SceneConst* c) {
    float lo[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
    float hi[3] = {-lo[0], -lo[1], -lo[2]};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nV;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float x = V[3 * i + a];
            lo[a] = fminf(lo[a], x);
            hi[a] = fmaxf(hi[a], x);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&c->lo_key[a], float_to_ordered(lo[a]));
            atomicMax(&c->hi_key[a], float_to_ordered(hi[a]));
        }
    }
}

__global__ void k_bounds_final(SceneConst* c, int64_t nV) {
    if (threadIdx.x != 0) return;
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        c->lo[a] = nV ? ordered_to_float(c->lo_key[a]) : 0.0f;
        c->hi[a] = nV ? ordered_to_float(c->hi_key[a]) : 0.0f;
        ext = fmaxf(ext, c->hi[a] - c->lo[a]);
    }
    c->eps = 1e-4f * ext;
}

// ---------------------------------------------------------------- morton
__device__ __forceinline__ uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Vertex index of corner k of triangle t, clamped into [0, nV) (and flagged)
// so that a bad index in the caller's F can never read out of bounds.
__device__ __forceinline__ int64_t corner(const int32_t* F, int64_t t, int k, int64_t nV,
                                          int32_t* status) {
    const int32_t i = F[3 * t + k];
    if (i < 0 || i >= nV) {
        atomicOr(status, FIPT_DEV_BAD_INDEX);
        return 0;
    }
    return i;
}

__global__ void k_morton(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ F,
                         int64_t T, const SceneConst* __restrict__ c, uint64_t* __restrict__ keys,
                         uint32_t* __restrict__ vals, int32_t* status) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    uint32_t q[3];
    const int64_t i0 = corner(F, t, 0, nV, status), i1 = corner(F, t, 1, nV, status),
                  i2 = corner(F, t, 2, nV, status);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x0 = V[3 * i0 + a], x1 = V[3 * i1 + a], x2 = V[3 * i2 + a];
        const float mn = fminf(fminf(x0, x1), x2), mx = fmaxf(fmaxf(x0, x1), x2);
        const double cc = __dmul_rn(0.5, __dadd_rn((double)mn, (double)mx));
        const double lo = (double)c->lo[a];
        const double ext = __dsub_rn((double)c->hi[a], lo);
        if (!(ext > 0.0)) {
            q[a] = 0;
            continue;
        }
        const double scale = __ddiv_rn(2097152.0, ext);
        double f = floor(__dmul_rn(__dsub_rn(cc, lo), scale));
        f = f < 0.0 ? 0.0 : (f > 2097151.0 ? 2097151.0 : f);
        q[a] = (uint32_t)f;
    }
    keys[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    vals[t] = (uint32_t)t;
}

// ---------------------------------------------------------------- karras
__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t x = k[i] ^ k[j];
    if (x) return __clzll((long long)x);
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_karras(const uint64_t* __restrict__ k, int64_t n, BvhNode* __restrict__ nodes,
                         int32_t* __restrict__ parent, int32_t* __restrict__ leaf_parent,
                         int32_t* __restrict__ range) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) > 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int64_t lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int64_t s = 0;
    int64_t div = 2;
    for (;;) {
        const int64_t t = (l + div - 1) / div;
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div <<= 1;
    }
    const int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    const int64_t first = i < j ? i : j, last = i < j ? j : i;
    const int c0 = (first == gamma) ? ~(int)gamma : (int)gamma;
    const int c1 = (last == gamma + 1) ? ~(int)(gamma + 1) : (int)(gamma + 1);
    nodes[i].d = make_int4(c0, c1, 0, 0);
    if (c0 >= 0) parent[c0] = (int)i; else leaf_parent[~c0] = (int)i;
    if (c1 >= 0) parent[c1] = (int)i; else leaf_parent[~c1] = (int)i;
    range[3 * i + 0] = (int)first;
    range[3 * i + 1] = (int)last;
    range[3 * i + 2] = (int)gamma;
    if (i == 0) parent[0] = -1;
}

// ---------------------------------------------------------------- pack
__global__ void k_pack(const float* __restrict__ V, int64_t nV, const int32_t* __restrict__ F,
                       const float* __restrict__ Le, const float* __restrict__ cache,
                       const uint32_t* __restrict__ sorted_idx, int64_t T, float4* __restrict__ tris,
                       float4* __restrict__ shade, int32_t* __restrict__ order, int32_t* status) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    const uint32_t t = sorted_idx[leaf];
    order[leaf] = (int32_t)t;
    const int64_t i0 = corner(F, t, 0, nV, status), i1 = corner(F, t, 1, nV, status),
                  i2 = corner(F, t, 2, nV, status);
    tris[3 * leaf + 0] = make_float4(V[3 * i0], V[3 * i0 + 1], V[3 * i0 + 2], __int_as_float((int)t));
    tris[3 * leaf + 1] = make_float4(V[3 * i1], V[3 * i1 + 1], V[3 * i1 + 2], 0.0f);
    tris[3 * leaf + 2] = make_float4(V[3 * i2], V[3 * i2 + 1], V[3 * i2 + 2], 0.0f);
    shade[2 * leaf + 0] = make_float4(Le[3 * t], Le[3 * t + 1], Le[3 * t + 2], 0.0f);
    shade[2 * leaf + 1] = make_float4(cache[3 * t], cache[3 * t + 1], cache[3 * t + 2], 0.0f);
}

__global__ void k_set_cache(const float* __restrict__ cache, const int32_t* __restrict__ order,
                            int64_t T, float4* __restrict__ shade) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    const int64_t t = order[leaf];
    shade[2 * leaf + 1] = make_float4(cache[3 * t], cache[3 * t + 1], cache[3 * t + 2], 0.0f);
}

// ---------------------------------------------------------------- emitters
__global__ void k_inverse(const int32_t* __restrict__ order, int64_t T, int32_t* __restrict__ inv) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf < T) inv[order[leaf]] = (int32_t)leaf;
}

// Emitter table for area sampling: emitter triangles (L_e > 0 in some
// channel) in original index order, their leaf, and cumulative areas in
// FP64 (areas from the packed float vertices in double).  k_emit_mark
// writes a 0/1 mark per triangle, an exclusive scan of the marks gives each
// emitter its position, k_emit_place writes leaf and area there, and one
// block turns the areas into the cumulative table and sets n_emit, A_emit.
__device__ __forceinline__ bool leaf_emits(const float4* shade, int leaf) {
    const float4 le = shade[2 * leaf];
    return le.x > 0.0f || le.y > 0.0f || le.z > 0.0f;
}

__global__ void k_emit_mark(const float4* __restrict__ shade, const int32_t* __restrict__ inv, int64_t T,
                            uint32_t* __restrict__ mark) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < T) mark[t] = leaf_emits(shade, inv[t]) ? 1u : 0u;
}

__global__ void k_emit_place(const float4* __restrict__ tris, const float4* __restrict__ shade,
                             const int32_t* __restrict__ inv, int64_t T, const uint32_t* __restrict__ pos,
                             int32_t* __restrict__ emit_leaf, double* __restrict__ emit_area) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= T) return;
    const int leaf = inv[t];
    if (!leaf_emits(shade, leaf)) return;
    const float4 p0 = tris[3 * leaf], p1 = tris[3 * leaf + 1], p2 = tris[3 * leaf + 2];
    const double e1[3] = {(double)p1.x - (double)p0.x, (double)p1.y - (double)p0.y, (double)p1.z - (double)p0.z};
    const double e2[3] = {(double)p2.x - (double)p0.x, (double)p2.y - (double)p0.y, (double)p2.z - (double)p0.z};
    const double cx = e1[1] * e2[2] - e1[2] * e2[1];
    const double cy = e1[2] * e2[0] - e1[0] * e2[2];
    const double cz = e1[0] * e2[1] - e1[1] * e2[0];
    emit_leaf[pos[t]] = leaf;
    emit_area[pos[t]] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
}

// In-place inclusive FP64 scan of the n_emit areas (n_emit = last position
// + last mark), one block walking them in chunks of 1024.
__global__ void __launch_bounds__(1024)
k_emit_cdf(const uint32_t* __restrict__ pos, const float4* __restrict__ shade, const int32_t* __restrict__ inv,
           int64_t T, double* __restrict__ cdf, SceneConst* c) {
    __shared__ double wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n = (int64_t)pos[T - 1] + (leaf_emits(shade, inv[T - 1]) ? 1 : 0);
    double carry = 0.0;
    for (int64_t base = 0; base < n; base += 1024) {
        const int64_t k = base + threadIdx.x;
        const double a = k < n ? cdf[k] : 0.0;
        double v = a;
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            double u = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const double y = __shfl_up_sync(0xffffffffu, u, o);
                if (lane >= o) u += y;
            }
            wsum[lane] = u;
        }
        __syncthreads();
        if (k < n) cdf[k] = carry + (warp > 0 ? wsum[warp - 1] : 0.0) + v;
        carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c->n_emit = (int)n;
        c->A_emit = carry;
    }
}

__global__ void k_set_materials(const float* __restrict__ albedo, const float* __restrict__ rough,
                                const float* __restrict__ metal, const int32_t* __restrict__ order,
                                int64_t T, float4* __restrict__ mats) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    const int64_t t = order[leaf];
    mats[2 * leaf] = make_float4(albedo[3 * t], albedo[3 * t + 1], albedo[3 * t + 2], rough[t]);
    mats[2 * leaf + 1] = make_float4(metal[t], 0.0f, 0.0f, 0.0f);
}

// ---------------------------------------------------------------- refit
struct Box {
    float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ Box leaf_box(const float4* tris, int leaf) {
    const float4 a = tris[3 * leaf], b = tris[3 * leaf + 1], c = tris[3 * leaf + 2];
    return Box{fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z),
               fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z)};
}

// Box of an internal node = union of its two child boxes, read through L2
// (written by another thread of this kernel before its fence + counter).
__device__ __forceinline__ Box node_box(const BvhNode* nodes, int i) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    const float4 a = __ldcg(p), b = __ldcg(p + 1), c = __ldcg(p + 2);
    return Box{fminf(a.x, b.x), fminf(a.z, b.z), fminf(c.x, c.z),
               fmaxf(a.y, b.y), fmaxf(a.w, b.w), fmaxf(c.y, c.w)};
}

__global__ void k_refit(BvhNode* nodes, const float4* __restrict__ tris,
                        const int32_t* __restrict__ parent, const int32_t* __restrict__ leaf_parent,
                        int32_t* flags, int64_t T) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    int p = leaf_parent[leaf];
    // a radix tree over 96-bit augmented keys is at most 97 levels deep
    for (int level = 0; p >= 0 && p < T - 1 && level < 128; ++level) {
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;   // the sibling finishes this node
        __threadfence();
        const int4 ch = __ldcg(reinterpret_cast<const int4*>(nodes + p) + 3);
        if ((ch.x < 0 ? (int64_t)~ch.x >= T : (int64_t)ch.x >= T - 1) ||
            (ch.y < 0 ? (int64_t)~ch.y >= T : (int64_t)ch.y >= T - 1))
            return;
        const Box b0 = ch.x < 0 ? leaf_box(tris, ~ch.x) : node_box(nodes, ch.x);
        const Box b1 = ch.y < 0 ? leaf_box(tris, ~ch.y) : node_box(nodes, ch.y);
        float4* q = reinterpret_cast<float4*>(nodes + p);
        __stcg(q + 0, make_float4(b0.lx, b0.hx, b0.ly, b0.hy));
        __stcg(q + 1, make_float4(b1.lx, b1.hx, b1.ly, b1.hy));
        __stcg(q + 2, make_float4(b0.lz, b0.hz, b1.lz, b1.hz));
        p = parent[p];
    }
}

// ---------------------------------------------------------------- treelets
// Treelet restructuring (Karras and Aila, HPG 2013) of the built tree.  A
// walk from every leaf climbs as in k_refit; when the second climb reaches
// an internal node p (its subtree is final), that thread's warp forms a
// treelet: p's two children,
// then, until there are TREELET leaves or only triangles, the treelet leaf
// with the largest surface area is replaced by its two children.  With one
// triangle per leaf the SAH cost of a topology differs from another's only
// in the areas of its internal nodes, so the optimal topology over the
// treelet's leaves minimises that sum; a dynamic programme over the 2^m - 1
// subsets finds it, and the treelet's internal nodes (p first, so p keeps
// its place under its parent) are rewritten when it is strictly cheaper.
// Leaves and their boxes are unchanged: the tree covers the same triangles
// with boxes as tight as before, and a closest-hit walk returns the same
// (t, triangle) minimum on any valid tree, up to near-ties that float32
// cannot separate (the culling bound depends on the visit order).
#ifndef FIPT_TREELET
#define FIPT_TREELET 7           // leaves per treelet: 2^7 - 1 subsets in the programme
#endif
constexpr int TREELET = FIPT_TREELET;
static_assert(TREELET >= 3 && TREELET <= 12, "treelets of 3 to 12 leaves");

__device__ __forceinline__ float half_area(const Box& b) {
    const float dx = fmaxf(b.hx - b.lx, 0.0f), dy = fmaxf(b.hy - b.ly, 0.0f), dz = fmaxf(b.hz - b.lz, 0.0f);
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ Box box_union(const Box& a, const Box& b) {
    return Box{fminf(a.lx, b.lx), fminf(a.ly, b.ly), fminf(a.lz, b.lz),
               fmaxf(a.hx, b.hx), fmaxf(a.hy, b.hy), fmaxf(a.hz, b.hz)};
}

// The two child boxes stored in node n's record (read through L2).
__device__ __forceinline__ void child_boxes(const BvhNode* nodes, int n, Box& b0, Box& b1, int4& ch) {
    const float4* q = reinterpret_cast<const float4*>(nodes + n);
    const float4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
    ch = __ldcg(reinterpret_cast<const int4*>(q + 3));
    b0 = Box{a.x, a.z, c.x, a.y, a.w, c.y};
    b1 = Box{b.x, b.z, c.z, b.y, b.w, c.w};
}

// Per-warp tables of the dynamic programme (shared memory).
struct TreeletTables {
    float area[1 << TREELET];
    float cost[1 << TREELET];
    uint16_t part[1 << TREELET];
};

// Restructures the treelet rooted at p; all 32 lanes of the warp call it
// with the same p.  Every lane forms the treelet (the same loads, served
// once), the lanes share the subsets of each size in the programme, and
// lane 0 writes the new internal nodes.
__device__ void restructure_warp(BvhNode* nodes, int32_t* parent, int32_t* leaf_parent, int p,
                                 TreeletTables& tb, int lane) {
    int ref[TREELET];
    Box box[TREELET];
    int inner[TREELET - 1];
    float area_l[TREELET];
    int m = 2, ni = 1;
    inner[0] = p;
    int4 ch;
    child_boxes(nodes, p, box[0], box[1], ch);
    ref[0] = ch.x;
    ref[1] = ch.y;
    area_l[0] = half_area(box[0]);
    area_l[1] = half_area(box[1]);
    float cur = half_area(box_union(box[0], box[1]));     // the current internal areas
#pragma unroll 1
    while (m < TREELET) {
        int best = -1;
        float ba = -1.0f;
        for (int i = 0; i < m; ++i)
            if (ref[i] >= 0 && area_l[i] > ba) {
                ba = area_l[i];
                best = i;
            }
        if (best < 0) break;
        const int n = ref[best];
        cur += ba;
        inner[ni++] = n;
        child_boxes(nodes, n, box[best], box[m], ch);
        ref[best] = ch.x;
        ref[m] = ch.y;
        area_l[best] = half_area(box[best]);
        area_l[m] = half_area(box[m]);
        ++m;
    }
    if (m < 3) return;                                     // two leaves have one topology (uniform)
    const int full = (1 << m) - 1;
    for (int S = lane + 1; S <= full; S += 32) {
        const int i0 = __ffs(S) - 1;
        Box b = box[i0];
        for (int i = i0 + 1; i < m; ++i)
            if (S & (1 << i)) b = box_union(b, box[i]);
        tb.area[S] = half_area(b);
        if ((S & (S - 1)) == 0) {
            tb.cost[S] = 0.0f;
            tb.part[S] = 0;
        }
    }
    __syncwarp();
    for (int k = 2; k <= m; ++k) {                         // subsets by size: smaller ones are done
        for (int S = lane + 1; S <= full; S += 32) {
            if (__popc(S) != k) continue;
            const int low = S & -S;
            float best = __int_as_float(0x7f800000);
            int bp = low;
            for (int P = (S - 1) & S; P > 0; P = (P - 1) & S) {
                if (!(P & low)) continue;
                const float v = tb.cost[P] + tb.cost[S ^ P];
                if (v < best) {
                    best = v;
                    bp = P;
                }
            }
            tb.cost[S] = best + tb.area[S];
            tb.part[S] = (uint16_t)bp;
        }
        __syncwarp();
    }
    if (lane == 0 && tb.cost[full] < cur * 0.99999f) {    // else keep the current topology
        // rebuild: depth-first from the full set; internal node k = inner[k]
        BvhNode rec[TREELET - 1];
        int stk_s[2 * TREELET], stk_par[2 * TREELET], stk_side[2 * TREELET];
        int sp = 0, next = 0;
        stk_s[sp] = full; stk_par[sp] = -1; stk_side[sp] = 0; ++sp;
        while (sp > 0) {
            --sp;
            const int S = stk_s[sp], par = stk_par[sp], side = stk_side[sp];
            int r;
            const int i0 = __ffs(S) - 1;
            Box b = box[i0];
            for (int i = i0 + 1; i < m; ++i)
                if (S & (1 << i)) b = box_union(b, box[i]);
            if ((S & (S - 1)) == 0) {
                r = ref[i0];
            } else {
                const int k = next++;
                r = inner[k];
                const int P = tb.part[S];
                stk_s[sp] = S ^ P; stk_par[sp] = k; stk_side[sp] = 1; ++sp;
                stk_s[sp] = P; stk_par[sp] = k; stk_side[sp] = 0; ++sp;
            }
            if (par >= 0) {
                BvhNode& R = rec[par];
                if (side == 0) {
                    R.a = make_float4(b.lx, b.hx, b.ly, b.hy);
                    R.c.x = b.lz; R.c.y = b.hz;
                    R.d.x = r;
                } else {
                    R.b = make_float4(b.lx, b.hx, b.ly, b.hy);
                    R.c.z = b.lz; R.c.w = b.hz;
                    R.d.y = r;
                }
                if (r >= 0) __stcg(parent + r, inner[par]);
                else __stcg(leaf_parent + ~r, inner[par]);
            }
        }
        for (int k = 0; k < ni; ++k) {
            rec[k].d.z = 0;
            rec[k].d.w = 0;
            float4* q = reinterpret_cast<float4*>(nodes + inner[k]);
            __stcg(q + 0, rec[k].a);
            __stcg(q + 1, rec[k].b);
            __stcg(q + 2, rec[k].c);
            __stcg(reinterpret_cast<int4*>(q + 3), rec[k].d);
        }
        __threadfence();
    }
    __syncwarp();
}

constexpr int TL_THREADS = 128;

// One restructuring pass.  flags[] must be zero.  Each thread climbs from
// its leaf; at every round the warp restructures, one after the other, the
// nodes its lanes were second to reach.  A climb longer than any valid
// tree allows (a corrupt parent chain) stops and raises the step flag.
__global__ void __launch_bounds__(TL_THREADS)
k_treelets(BvhNode* nodes, int32_t* parent, int32_t* leaf_parent, int32_t* flags, int64_t T, int32_t* status) {
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ TreeletTables tabs[TL_THREADS / 32];
    TreeletTables& tb = tabs[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t leaf = blockIdx.x * (int64_t)TL_THREADS + threadIdx.x;
    int p = leaf < T ? __ldcg(leaf_parent + leaf) : -1;
    bool act = p >= 0 && p < T - 1;
    int level = 0;
    for (;;) {
        if (act) {
            if (++level > 4096) {
                atomicOr(status, FIPT_DEV_STEP_LIMIT);
                act = false;
            } else {
                __threadfence();
                if (atomicAdd(&flags[p], 1) == 0) act = false;   // the other child's climb goes on
                __threadfence();
            }
        }
        unsigned todo = __ballot_sync(FULL, act);
        if (todo == 0) break;
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            restructure_warp(nodes, parent, leaf_parent, __shfl_sync(FULL, p, l), tb, lane);
        }
        if (act) {
            __threadfence();
            p = __ldcg(parent + p);
            act = p >= 0 && p < T - 1;
        }
    }
}

// ---------------------------------------------------------------- relayout
// Depth-first renumbering of the internal nodes: the root stays 0, a node's
// first child follows it, its second child follows the first child's
// subtree.  Walks descend into the first child most of the time and
// subtrees occupy contiguous records, so a walk's records share cache lines
// more often.  The topology, child order and boxes are unchanged: every walk
// visits the same nodes in the same order as before, on new addresses.

// Internal nodes in every subtree (a climb as in k_refit; flags zeroed).
__global__ void k_subtree_sizes(const BvhNode* nodes, const int32_t* parent, const int32_t* leaf_parent,
                                int32_t* flags, int32_t* size, int64_t T, int32_t* status) {
    const int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (leaf >= T) return;
    int p = __ldcg(leaf_parent + leaf);
    for (int level = 0; p >= 0 && p < T - 1; ++level) {
        if (level >= 4096) {
            atomicOr(status, FIPT_DEV_STEP_LIMIT);
            return;
        }
        __threadfence();
        if (atomicAdd(&flags[p], 1) == 0) return;          // the other child's climb goes on
        __threadfence();
        const int4 ch = __ldcg(reinterpret_cast<const int4*>(nodes + p) + 3);
        const int s0 = (ch.x >= 0 && ch.x < T - 1) ? __ldcg(size + ch.x) : 0;
        const int s1 = (ch.y >= 0 && ch.y < T - 1) ? __ldcg(size + ch.y) : 0;
        __stcg(size + p, s0 + s1 + 1);
        __threadfence();
        p = __ldcg(parent + p);
    }
}

// Depth-first index of every internal node: the sum, over the path from
// the root, of 1 per step plus the first child's subtree size where the
// path takes the second child.
__global__ void k_dfs_index(const BvhNode* __restrict__ nodes, const int32_t* __restrict__ parent,
                            const int32_t* __restrict__ size, int32_t* __restrict__ idx, int64_t n,
                            int32_t* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cur = (int)i, pos = 0;
    for (int level = 0; cur != 0; ++level) {
        const int p = cur > 0 && cur < n ? parent[cur] : -1;
        if (level >= 4096 || p < 0 || p >= n) {
            atomicOr(status, FIPT_DEV_STEP_LIMIT);
            idx[i] = -1;
            return;
        }
        const int4 ch = __ldg(reinterpret_cast<const int4*>(nodes + p) + 3);
        pos += (cur == ch.y && ch.x >= 0 && ch.x < n) ? 1 + size[ch.x] : 1;
        cur = p;
    }
    idx[i] = pos;
}

// Writes node i's record at idx[i] with renumbered child and parent links.
__global__ void k_relabel(const BvhNode* __restrict__ nodes, const int32_t* __restrict__ parent,
                          const int32_t* __restrict__ idx, BvhNode* __restrict__ out,
                          int32_t* __restrict__ out_parent, int64_t n, int32_t* status) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = idx[i];
    if (j < 0 || j >= n) {
        atomicOr(status, FIPT_DEV_BAD_NODE);
        return;
    }
    BvhNode r = nodes[i];
    if (r.d.x >= 0) r.d.x = r.d.x < n ? idx[r.d.x] : r.d.x;
    if (r.d.y >= 0) r.d.y = r.d.y < n ? idx[r.d.y] : r.d.y;
    out[j] = r;
    const int p = parent[i];
    out_parent[j] = (p >= 0 && p < n) ? idx[p] : -1;
}

__global__ void k_relabel_leaves(int32_t* leaf_parent, const int32_t* __restrict__ idx, int64_t T, int64_t n) {
    const int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (l >= T) return;
    const int p = leaf_parent[l];
    if (p >= 0 && p < n) leaf_parent[l] = idx[p];
}

// One-triangle scene: a root whose first child is leaf 0 and whose second
// child has an empty box.
__global__ void k_single(BvhNode* nodes, const float4* __restrict__ tris, int32_t* range) {
    const Box b = leaf_box(tris, 0);
    const float inf = __int_as_float(0x7f800000);
    nodes[0].a = make_float4(b.lx, b.hx, b.ly, b.hy);
    nodes[0].b = make_float4(inf, -inf, inf, -inf);
    nodes[0].c = make_float4(b.lz, b.hz, inf, -inf);
    nodes[0].d = make_int4(~0, ~0, 0, 0);
    range[0] = 0; range[1] = 0; range[2] = 0;
}

__global__ void k_export_boxes(const BvhNode* __restrict__ nodes, int64_t n, float* __restrict__ out,
                               int32_t* __restrict__ child) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const BvhNode nd = nodes[i];
    if (child) {
        child[2 * i] = nd.d.x;
        child[2 * i + 1] = nd.d.y;
    }
    if (!out) return;
    out[6 * i + 0] = fminf(nd.a.x, nd.b.x);
    out[6 * i + 1] = fminf(nd.a.z, nd.b.z);
    out[6 * i + 2] = fminf(nd.c.x, nd.c.z);
    out[6 * i + 3] = fmaxf(nd.a.y, nd.b.y);
    out[6 * i + 4] = fmaxf(nd.a.w, nd.b.w);
    out[6 * i + 5] = fmaxf(nd.c.y, nd.c.w);
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------- sort driver
// Histogram (RADIX x blocks, digit-major) followed, 256-byte aligned, by the
// chunk sums of the multi-block scan.
static int64_t hist_words(int64_t n) {
    const int64_t m = (int64_t)RADIX * (sort_blocks(n) > 0 ? sort_blocks(n) : 1);
    return (m + 63) & ~int64_t(63);
}

size_t radix_sort_scratch_bytes(int64_t n) {
    const int64_t m = hist_words(n);
    return (size_t)(m + (m + SCAN_CHUNK - 1) / SCAN_CHUNK + 64) * sizeof(uint32_t);
}

// Exclusive scan of the m = RADIX * nb histogram counters.
static fipt_status scan_hist(uint32_t* hist, int64_t m, uint32_t* bsum, cudaStream_t st) {
    if (m <= 4 * SCAN_CHUNK) {
        FIPT_LAUNCH(k_scan_single, 1, SCAN_THREADS, 0, st, hist, m);
        return FIPT_OK;
    }
    const int64_t nc = (m + SCAN_CHUNK - 1) / SCAN_CHUNK;
    FIPT_LAUNCH(k_scan_reduce, (unsigned)nc, SCAN_THREADS, 0, st, hist, m, bsum);
    FIPT_LAUNCH(k_scan_single, 1, SCAN_THREADS, 0, st, bsum, nc);
    FIPT_LAUNCH(k_scan_apply, (unsigned)nc, SCAN_THREADS, 0, st, hist, m, bsum);
    return FIPT_OK;
}

template <class K>
fipt_status radix_sort_pairs(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                             uint32_t* hist, int64_t n, int bits, cudaStream_t st, K** out_keys,
                             uint32_t** out_vals, const uint32_t* n_dev) {
    K *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    const int64_t nb = sort_blocks(n);
    if (n > 0) {
        for (int shift = 0; shift < bits; shift += 8) {
            FIPT_LAUNCH(k_sort_hist<K>, (unsigned)nb, SORT_THREADS, 0, st, ka, n, n_dev, shift, hist);
            fipt_status r = scan_hist(hist, (int64_t)RADIX * nb, hist + hist_words(n), st);
            if (r != FIPT_OK) return r;
            FIPT_LAUNCH(k_sort_scatter<K>, (unsigned)nb, SORT_THREADS, 0, st, ka, va, kb, vb, n, n_dev, shift,
                        hist);
            K* tk = ka; ka = kb; kb = tk;
            uint32_t* tv = va; va = vb; vb = tv;
        }
        FIPT_LAUNCHED("radix sort");
    }
    *out_keys = ka;
    *out_vals = va;
    return FIPT_OK;
}

template fipt_status radix_sort_pairs<uint64_t>(uint64_t*, uint64_t*, uint32_t*, uint32_t*,
                                                uint32_t*, int64_t, int, cudaStream_t,
                                                uint64_t**, uint32_t**, const uint32_t*);
template fipt_status radix_sort_pairs<uint32_t>(uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                                uint32_t*, int64_t, int, cudaStream_t,
                                                uint32_t**, uint32_t**, const uint32_t*);

fipt_status rebuild_emitter_table(fipt_scene* s, cudaStream_t st) {
    if (s->T == 0) return FIPT_OK;
    const int64_t T = s->T;
    // the sort scratch (values, histogram) is free once the tree is built
    FIPT_LAUNCH(k_emit_mark, grid_for(T, 256), 256, 0, st, s->shade, s->inv, T, s->vals);
    fipt_status r = scan_hist(s->vals, T, s->hist, st);
    if (r != FIPT_OK) return r;
    FIPT_LAUNCH(k_emit_place, grid_for(T, 256), 256, 0, st, s->tris, s->shade, s->inv, T, s->vals,
                s->emit_leaf, s->emit_cdf);
    FIPT_LAUNCH(k_emit_cdf, 1, 1024, 0, st, s->vals, s->shade, s->inv, T, s->emit_cdf, s->cst);
    FIPT_LAUNCHED("emitter table");
    return FIPT_OK;
}

// ---------------------------------------------------------------- C ABI
namespace {
struct SceneLayout {
    SceneConst* cst;
    BvhNode* nodes;
    BvhNode* nodes_alt;     // the relayout's target
    int32_t* scratch;       // [3 (T-1)] subtree sizes, new indices, new parents
    float4* tris;
    float4* shade;
    int32_t* order;
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt, *hist;
    int32_t *range, *parent, *leaf_parent, *flags;
    float4* mats;
    int32_t *inv, *emit_leaf;
    double* emit_cdf;
    size_t bytes;
};

SceneLayout carve_scene(void* ws, int64_t T) {
    Carver c{static_cast<char*>(ws), 0};
    SceneLayout L;
    const int64_t ni = T > 1 ? T - 1 : 1;
    const int64_t t1 = T > 0 ? T : 1;
    L.cst = c.take<SceneConst>(1);
    L.nodes = c.take<BvhNode>((size_t)ni);
    L.nodes_alt = c.take<BvhNode>((size_t)ni);
    L.scratch = c.take<int32_t>((size_t)(3 * ni));
    L.tris = c.take<float4>((size_t)(3 * t1));
    L.shade = c.take<float4>((size_t)(2 * t1));
    L.order = c.take<int32_t>((size_t)t1);
    L.keys = c.take<uint64_t>((size_t)t1);
    L.keys_alt = c.take<uint64_t>((size_t)t1);
    L.vals = c.take<uint32_t>((size_t)t1);
    L.vals_alt = c.take<uint32_t>((size_t)t1);
    L.hist = c.take<uint32_t>(radix_sort_scratch_bytes(t1) / sizeof(uint32_t));
    L.range = c.take<int32_t>((size_t)(3 * ni));
    L.parent = c.take<int32_t>((size_t)ni);
    L.leaf_parent = c.take<int32_t>((size_t)t1);
    L.flags = c.take<int32_t>((size_t)ni);
    L.mats = c.take<float4>((size_t)(2 * t1));
    L.inv = c.take<int32_t>((size_t)t1);
    L.emit_leaf = c.take<int32_t>((size_t)t1);
    L.emit_cdf = c.take<double>((size_t)t1);
    L.bytes = c.off + 256;
    return L;
}
}  // namespace

extern "C" fipt_status fipt_scene_workspace_size(int64_t nV, int64_t T, size_t* bytes) {
    FIPT_REQUIRE(bytes, "bytes is NULL");
    FIPT_REQUIRE(nV >= 0 && T >= 0 && T < (int64_t)1 << 31, "bad sizes nV=%lld T=%lld",
                 (long long)nV, (long long)T);
    *bytes = carve_scene(nullptr, T).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_create(fipt_ctx* ctx, const float* V, int64_t nV,
                                         const int32_t* F, int64_t T, const float* Le,
                                         const float* cache, void* workspace, size_t ws_bytes,
                                         fipt_stream stream, fipt_scene** out) {
    FIPT_REQUIRE(ctx && out, "ctx / out is NULL");
    FIPT_REQUIRE(nV >= 0 && T >= 0 && T < (int64_t)1 << 31, "bad sizes nV=%lld T=%lld",
                 (long long)nV, (long long)T);
    FIPT_REQUIRE(T == 0 || (V && F && Le && cache), "V / F / Le / cache is NULL");
    FIPT_REQUIRE(T == 0 || nV > 0, "triangles without vertices");
    FIPT_REQUIRE(fipt_aligned(V, 4) && fipt_aligned(F, 4) && fipt_aligned(Le, 4) &&
                 fipt_aligned(cache, 4), "inputs must be 4-byte aligned");
    FIPT_REQUIRE(workspace && fipt_aligned(workspace, 256), "workspace must be 256-byte aligned");
    SceneLayout L = carve_scene(workspace, T);
    if (ws_bytes < L.bytes)
        return fipt_set_error(FIPT_ERR_WORKSPACE, "scene workspace %zu < %zu bytes", ws_bytes, L.bytes);
    FIPT_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    fipt_scene* s = new fipt_scene();
    s->ctx = ctx; s->nV = nV; s->T = T;
    s->cst = L.cst; s->nodes = L.nodes; s->tris = L.tris; s->shade = L.shade; s->order = L.order;
    s->keys = L.keys; s->keys_alt = L.keys_alt; s->vals = L.vals; s->vals_alt = L.vals_alt;
    s->hist = L.hist; s->range = L.range; s->parent = L.parent; s->leaf_parent = L.leaf_parent;
    s->flags = L.flags; s->ws_bytes = L.bytes;
    s->mats = L.mats; s->inv = L.inv; s->emit_leaf = L.emit_leaf; s->emit_cdf = L.emit_cdf;
    s->nodes_alt = L.nodes_alt; s->scratch = L.scratch;

    FIPT_LAUNCH(k_bounds_init, 1, 32, 0, st, L.cst);
    if (nV > 0) {
        const int64_t nb = (nV + 255) / 256;
        FIPT_LAUNCH(k_bounds, (unsigned)(nb < 1216 ? nb : 1216), 256, 0, st, V, nV, L.cst);
    }
    FIPT_LAUNCH(k_bounds_final, 1, 32, 0, st, L.cst, nV);
    if (T > 0) {
        FIPT_LAUNCH(k_morton, grid_for(T, 256), 256, 0, st, V, nV, F, T, L.cst, L.keys, L.vals,
                    ctx->status);
        uint64_t* sk;
        uint32_t* sv;
        fipt_status r = radix_sort_pairs<uint64_t>(L.keys, L.keys_alt, L.vals, L.vals_alt, L.hist,
                                                   T, 64, st, &sk, &sv);
        if (r != FIPT_OK) { delete s; return r; }
        s->keys = sk;   // 8 passes: the result is back in the first buffer
        FIPT_LAUNCH(k_pack, grid_for(T, 256), 256, 0, st, V, nV, F, Le, cache, sv, T, L.tris, L.shade,
                    L.order, ctx->status);
        if (T == 1) {
            FIPT_LAUNCH(k_single, 1, 1, 0, st, L.nodes, L.tris, L.range);
        } else {
            FIPT_LAUNCH(k_karras, grid_for(T - 1, 256), 256, 0, st, sk, T, L.nodes, L.parent,
                                                           L.leaf_parent, L.range);
            cudaError_t e = cudaMemsetAsync(L.flags, 0, sizeof(int32_t) * (size_t)(T - 1), st);
            if (e != cudaSuccess) { delete s; return fipt_check_cuda(e, "memset flags"); }
            FIPT_LAUNCH(k_refit, grid_for(T, 256), 256, 0, st, L.nodes, L.tris, L.parent, L.leaf_parent,
                                                      L.flags, T);
        }
        FIPT_LAUNCH(k_inverse, grid_for(T, 256), 256, 0, st, L.order, T, L.inv);
        fipt_status re = rebuild_emitter_table(s, st);
        if (re != FIPT_OK) { delete s; return re; }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { delete s; return fipt_check_cuda(e, "scene build"); }
    *out = s;
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_optimize(fipt_scene* s, int32_t passes, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(passes >= 0 && passes <= 16, "passes must be in [0, 16]");
    const int64_t T = s->T;
    if (T < 3 || passes == 0) return FIPT_OK;
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int k = 0; k < passes; ++k) {
        FIPT_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * (size_t)(T - 1), st));
        FIPT_LAUNCH(k_treelets, grid_for(T, TL_THREADS), TL_THREADS, 0, st, s->nodes, s->parent, s->leaf_parent, s->flags, T,
                    s->ctx->status);
    }
    FIPT_LAUNCHED("treelet restructuring");
    s->restructured = true;
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_relayout(fipt_scene* s, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    const int64_t T = s->T, n = T - 1;
    if (T < 3) return FIPT_OK;
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t* size = s->scratch;
    int32_t* idx = s->scratch + n;
    int32_t* new_parent = s->scratch + 2 * n;
    FIPT_CUDA(cudaMemsetAsync(s->flags, 0, sizeof(int32_t) * (size_t)n, st));
    FIPT_LAUNCH(k_subtree_sizes, grid_for(T, 256), 256, 0, st, s->nodes, s->parent, s->leaf_parent, s->flags, size,
                T, s->ctx->status);
    FIPT_LAUNCH(k_dfs_index, grid_for(n, 256), 256, 0, st, s->nodes, s->parent, size, idx, n, s->ctx->status);
    FIPT_LAUNCH(k_relabel, grid_for(n, 256), 256, 0, st, s->nodes, s->parent, idx, s->nodes_alt, new_parent, n,
                s->ctx->status);
    FIPT_LAUNCH(k_relabel_leaves, grid_for(T, 256), 256, 0, st, s->leaf_parent, idx, T, n);
    FIPT_LAUNCHED("relayout");
    BvhNode* t = s->nodes;
    s->nodes = s->nodes_alt;
    s->nodes_alt = t;
    FIPT_CUDA(cudaMemcpyAsync(s->parent, new_parent, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, st));
    s->restructured = true;
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_set_cache(fipt_scene* s, const float* cache, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(s->T == 0 || (cache && fipt_aligned(cache, 4)), "cache is NULL or misaligned");
    if (s->T == 0) return FIPT_OK;
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    FIPT_LAUNCH(k_set_cache, grid_for(s->T, 256), 256, 0, static_cast<cudaStream_t>(stream), cache, s->order, s->T, s->shade);
    FIPT_LAUNCHED("set cache");
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_destroy(fipt_scene* s) {
    delete s;
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_info(fipt_scene* s, fipt_stream stream, int64_t* T, float* eps,
                                       float* lo3, float* hi3) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    SceneConst c;
    FIPT_CUDA(cudaMemcpyAsync(&c, s->cst, sizeof(c), cudaMemcpyDeviceToHost,
                              static_cast<cudaStream_t>(stream)));
    FIPT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    if (T) *T = s->T;
    if (eps) *eps = c.eps;
    for (int a = 0; a < 3; ++a) {
        if (lo3) lo3[a] = c.lo[a];
        if (hi3) hi3[a] = c.hi[a];
    }
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_debug_export(fipt_scene* s, uint64_t* morton, int32_t* order,
                                               int32_t* node_range, float* node_box, int32_t* node_child,
                                               fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t T = s->T, ni = T > 1 ? T - 1 : (T == 1 ? 1 : 0);
    if (T == 0) return FIPT_OK;
    if (morton) FIPT_CUDA(cudaMemcpyAsync(morton, s->keys, 8 * (size_t)T, cudaMemcpyDeviceToDevice, st));
    if (order) FIPT_CUDA(cudaMemcpyAsync(order, s->order, 4 * (size_t)T, cudaMemcpyDeviceToDevice, st));
    FIPT_REQUIRE(!(node_range && s->restructured),
                 "the tree was restructured: its nodes no longer match the radix-tree ranges");
    if (node_range)
        FIPT_CUDA(cudaMemcpyAsync(node_range, s->range, 12 * (size_t)ni, cudaMemcpyDeviceToDevice, st));
    if (node_box || node_child) {
        FIPT_LAUNCH(k_export_boxes, grid_for(ni, 256), 256, 0, st, s->nodes, ni, node_box, node_child);
        FIPT_LAUNCHED("export boxes");
    }
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_set_materials(fipt_scene* s, const float* albedo, const float* rough,
                                                const float* metal, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(s->T == 0 || (albedo && rough && metal), "material array is NULL");
    FIPT_REQUIRE(fipt_aligned(albedo, 4) && fipt_aligned(rough, 4) && fipt_aligned(metal, 4),
                 "materials must be 4-byte aligned");
    s->has_materials = true;
    if (s->T == 0) return FIPT_OK;
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    FIPT_LAUNCH(k_set_materials, grid_for(s->T, 256), 256, 0, static_cast<cudaStream_t>(stream),
                albedo, rough, metal, s->order, s->T, s->mats);
    FIPT_LAUNCHED("set materials");
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_set_environment(fipt_scene* s, const float* env, int32_t W,
                                                  int32_t H) {
    FIPT_REQUIRE(s, "scene is NULL");
    if (!env) {
        s->env = nullptr;
        s->env_w = s->env_h = 0;
        return FIPT_OK;
    }
    FIPT_REQUIRE(W > 0 && H > 0, "environment size must be positive");
    FIPT_REQUIRE(fipt_aligned(env, 4), "environment map must be 4-byte aligned");
    s->env = env;
    s->env_w = W;
    s->env_h = H;
    return FIPT_OK;
}
