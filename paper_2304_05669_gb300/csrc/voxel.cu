// Voxel radiance cache (Sec. 4.2): the input pixels' radiance is
// average-pooled onto an R^3 grid spanned over the scene box and queried at
// the voxel containing a hit point (the paper uses R = 256).  Pixels are
// assigned to voxels as correctly rounded FP64 operations place them (as
// the Morton quantisation), grouped by a stable radix sort on the voxel
// index, and each voxel's mean is its FP64 sum in pixel order over the
// count, so the grid is deterministic.  GB300 runs FP64 at 1/64 of the
// float32 rate, so both steps reach those FP64 results by cheaper exact
// means: cells in float32 away from cell faces, sums in integers while
// they are provably exact (k_vox_keys, k_vox_means), FP64 otherwise.
#include "fipt_internal.cuh"
#include "exact_sum.cuh"

namespace {

// The per-axis scale R / (hi - lo) is the same correctly rounded double for
// every pixel; the first three threads of a block compute it once.
//
// A pixel's cell on an axis is floor(RN64(RN64(x - lo) * scale)), clamped
// to [0, R - 1].  Most cells are found in float32 without changing that
// result: f = RN32(RN32(x - lo) * RN32(scale)) and the FP64 value both lie
// within relative 2^-24 (three roundings) plus 2^-53 (two) of the exact
// product, so |f - f64| < 2^-22 |f| away from underflow.  When no integer
// in [1, R - 1] lies within 2^-21 |f| of f, no cell face separates f from
// the FP64 value and floor(f) clamps to the same cell; a cell face at 0 or
// R clamps either side to the same cell, and an f that underflows keeps
// the sign of x - lo.  Pixels near an inner cell face (and NaNs) take the
// FP64 arithmetic, and so does every pixel on an axis whose float32 scale
// is infinite or subnormal (extents below ~1e-35 or near 1e38), where the
// bound does not hold.
__global__ void k_vox_keys(const float* __restrict__ x, int64_t stride, int64_t P,
                           const SceneConst* __restrict__ c, int R, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    __shared__ double scale[3];
    __shared__ float scale32[3];
    __shared__ bool fast[3];
    if (threadIdx.x < 3) {
        const double ext = __dsub_rn((double)c->hi[threadIdx.x], (double)c->lo[threadIdx.x]);
        scale[threadIdx.x] = ext > 0.0 ? __ddiv_rn((double)R, ext) : 0.0;
        const float s32 = __double2float_rn(scale[threadIdx.x]);
        scale32[threadIdx.x] = s32;
        fast[threadIdx.x] = s32 == 0.0f || (s32 >= 1.17549435e-38f && s32 <= 3.40282347e38f);
    }
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    uint32_t ix[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xa = x[p * stride + a];
        const float lo32 = c->lo[a];
        const float f = __fmul_rn(__fsub_rn(xa, lo32), scale32[a]);
        const float r = rintf(f);
        const bool near_face = r >= 1.0f && r <= (float)(R - 1) && fabsf(f - r) <= fabsf(f) * 0x1p-21f;
        if (fast[a] && !near_face && f == f) {
            const float fl = floorf(f);
            ix[a] = fl < 0.0f ? 0u : (fl > (float)(R - 1) ? (uint32_t)(R - 1) : (uint32_t)fl);
        } else {
            const double lo = (double)lo32;
            double g = 0.0;
            if (scale[a] > 0.0) g = __dmul_rn(__dsub_rn((double)xa, lo), scale[a]);
            double fl = floor(g);
            fl = fl < 0.0 ? 0.0 : (fl > (double)(R - 1) ? (double)(R - 1) : fl);
            ix[a] = (uint32_t)fl;
        }
    }
    keys[p] = (ix[2] * (uint32_t)R + ix[1]) * (uint32_t)R + ix[0];
    vals[p] = (uint32_t)p;
}

// Run heads (the first sorted pixel of each voxel's run) listed in pixel
// order, so that run h spans [heads[h], heads[h + 1]) with heads[nh] = P:
// k_vox_count counts the heads of each tile of HEAD_TILE pixels,
// k_vox_scan turns the counts into offsets (one block) and k_vox_compact
// writes each tile's heads at its offset.
constexpr int HEAD_TILE = 1024;

__device__ __forceinline__ bool run_head(const uint32_t* __restrict__ keys, int64_t j, int64_t P) {
    return j < P && (j == 0 || keys[j - 1] != keys[j]);
}

// Exclusive prefix of v over the block's 32 warps (v given by lane 0 of
// each warp in ws[w]); ws[w] becomes the sum of warps before w and the
// return value (all threads) the block total.
__device__ __forceinline__ uint32_t warp_offsets(uint32_t* ws) {
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const uint32_t v = ws[lane];
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        ws[lane] = x - v;
        if (lane == 31) ws[32] = x;
    }
    __syncthreads();
    return ws[32];
}

__global__ void __launch_bounds__(HEAD_TILE)
k_vox_count(const uint32_t* __restrict__ keys, int64_t P, uint32_t* __restrict__ tcount) {
    __shared__ uint32_t ws[33];
    const int64_t j = blockIdx.x * (int64_t)HEAD_TILE + threadIdx.x;
    const unsigned m = __ballot_sync(0xffffffffu, run_head(keys, j, P));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = __popc(m);
    const uint32_t total = warp_offsets(ws);
    if (threadIdx.x == 0) tcount[blockIdx.x] = total;
}

// One block: exclusive scan of the nt tile counts in place, nh = their sum,
// heads[nh] = P.
__global__ void __launch_bounds__(HEAD_TILE)
k_vox_scan(uint32_t* __restrict__ tcount, int64_t nt, uint32_t* __restrict__ heads, uint32_t* __restrict__ nhead,
           int64_t P) {
    __shared__ uint32_t ws[33];
    const int lane = threadIdx.x & 31;
    uint32_t carry = 0;
    for (int64_t base = 0; base < nt; base += HEAD_TILE) {
        const int64_t i = base + threadIdx.x;
        const uint32_t v = i < nt ? tcount[i] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[threadIdx.x >> 5] = x;
        const uint32_t total = warp_offsets(ws);
        if (i < nt) tcount[i] = carry + ws[threadIdx.x >> 5] + x - v;
        carry += total;
        __syncthreads();                         // ws is rewritten by the next chunk
    }
    if (threadIdx.x == 0) {
        *nhead = carry;
        heads[carry] = (uint32_t)P;
    }
}

__global__ void __launch_bounds__(HEAD_TILE)
k_vox_compact(const uint32_t* __restrict__ keys, int64_t P, const uint32_t* __restrict__ toff,
              uint32_t* __restrict__ heads) {
    __shared__ uint32_t ws[33];
    const int lane = threadIdx.x & 31;
    const int64_t j = blockIdx.x * (int64_t)HEAD_TILE + threadIdx.x;
    const bool h = run_head(keys, j, P);
    const unsigned m = __ballot_sync(0xffffffffu, h);
    if (lane == 0) ws[threadIdx.x >> 5] = __popc(m);
    warp_offsets(ws);
    if (h) heads[toff[blockIdx.x] + ws[threadIdx.x >> 5] + __popc(m & ((1u << lane) - 1u))] = (uint32_t)j;
}

#ifndef FIPT_VOX_THREADS
#define FIPT_VOX_THREADS 64      // small blocks: a long run holds few other runs' slots
#endif
#ifndef FIPT_VOX_UNROLL
#define FIPT_VOX_UNROLL 8        // pixels per group
#endif
constexpr int MEAN_THREADS = FIPT_VOX_THREADS;
constexpr int VU = FIPT_VOX_UNROLL;

// A thread per voxel run: the run's pixels are taken VU at a time, the next
// group's pixel indices loading while this group's radiance is fetched, and
// each channel's FP64 sum in pixel order is carried exactly in integers
// (exact_sum.cuh) while the run's exponent range allows it.  emin and emax
// are tracked over the three channels together, and the sums are rescaled
// when a group brings a smaller exponent.  A run that leaves the exact range
// is summed again with FP64 additions in pixel order.
__global__ void __launch_bounds__(MEAN_THREADS)
k_vox_means(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ pix, const uint32_t* __restrict__ heads,
            const uint32_t* __restrict__ nhead, const float* __restrict__ L, float4* __restrict__ grid) {
    const int64_t nh = *nhead;
    for (int64_t h = blockIdx.x * (int64_t)MEAN_THREADS + threadIdx.x; h < nh;
         h += (int64_t)gridDim.x * MEAN_THREADS) {
        const int64_t j0 = heads[h], j1 = heads[h + 1];
        const uint32_t k = keys[j0];
        long long acc[3] = {0, 0, 0};
        int emin = fipt_exact::EMPTY_EMIN;
        fipt_exact::Range run;
        bool ok = fipt_exact::spread_limit(j1 - j0) >= 0;
        uint32_t qn[VU];
#pragma unroll
        for (int u = 0; u < VU; ++u) qn[u] = j0 + u < j1 ? pix[j0 + u] : 0u;
        for (int64_t e = j0; e < j1 && ok; e += VU) {
            float v[VU][3];
#pragma unroll
            for (int u = 0; u < VU; ++u) {
                const int64_t q = 3 * (int64_t)qn[u];
                const bool in = e + u < j1;
                v[u][0] = in ? L[q] : 0.0f;
                v[u][1] = in ? L[q + 1] : 0.0f;
                v[u][2] = in ? L[q + 2] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < VU; ++u) qn[u] = e + VU + u < j1 ? pix[e + VU + u] : 0u;
#pragma unroll
            for (int u = 0; u < VU; ++u)
#pragma unroll
                for (int c = 0; c < 3; ++c) run.note(v[u][c]);
            const int em = run.emin();
            if (em < emin) {            // from EMPTY_EMIN the sums are still 0
                const int sh = min(emin - em, 63);
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] = (long long)((unsigned long long)acc[c] << sh);
                emin = em;
            }
            ok = !run.special() && run.exact_for(j1 - j0);
            if (ok) {
#pragma unroll
                for (int u = 0; u < VU; ++u)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[c] += fipt_exact::term(v[u][c], emin);
            }
        }
        double s0, s1, s2;
        if (ok) {
            s0 = fipt_exact::scaled_double(acc[0], emin);
            s1 = fipt_exact::scaled_double(acc[1], emin);
            s2 = fipt_exact::scaled_double(acc[2], emin);
        } else {
            s0 = s1 = s2 = 0.0;
            for (int64_t e = j0; e < j1; ++e) {
                const int64_t q = 3 * (int64_t)pix[e];
                s0 += (double)L[q];
                s1 += (double)L[q + 1];
                s2 += (double)L[q + 2];
            }
        }
        const double n = (double)(j1 - j0);
        grid[k] = make_float4((float)(s0 / n), (float)(s1 / n), (float)(s2 / n), (float)n);
    }
}

struct VoxLayout {
    uint32_t *keys, *keys_alt, *vals, *vals_alt, *hist, *heads, *nhead, *tcount;
    size_t bytes;
};

VoxLayout carve(void* ws, int64_t P) {
    Carver c{static_cast<char*>(ws), 0};
    VoxLayout L;
    const int64_t p1 = P > 0 ? P : 1;
    L.keys = c.take<uint32_t>((size_t)p1);
    L.keys_alt = c.take<uint32_t>((size_t)p1);
    L.vals = c.take<uint32_t>((size_t)p1);
    L.vals_alt = c.take<uint32_t>((size_t)p1);
    L.hist = c.take<uint32_t>(radix_sort_scratch_bytes(p1) / sizeof(uint32_t));
    L.heads = c.take<uint32_t>((size_t)p1 + 1);
    L.nhead = c.take<uint32_t>(1);
    L.tcount = c.take<uint32_t>((size_t)((p1 + HEAD_TILE - 1) / HEAD_TILE));
    L.bytes = c.off + 256;
    return L;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" fipt_status fipt_voxel_cache_workspace_size(int64_t P, size_t* bytes) {
    FIPT_REQUIRE(bytes && P >= 0 && P < ((int64_t)1 << 31), "bad arguments");
    *bytes = carve(nullptr, P).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_voxel_cache_build(fipt_scene* s, const float* x, int64_t x_stride,
                                              const float* L, int64_t P, int32_t R, float* grid,
                                              void* ws, size_t ws_bytes, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(R >= 1 && R <= 1024, "R must be in [1, 1024]");
    FIPT_REQUIRE(P >= 0 && P < ((int64_t)1 << 31) && x_stride >= 3, "bad sizes");
    FIPT_REQUIRE(grid && fipt_aligned(grid, 16), "grid must be 16-byte aligned");
    FIPT_REQUIRE(P == 0 || (x && L && fipt_aligned(x, 4) && fipt_aligned(L, 4)), "x / L NULL or misaligned");
    VoxLayout Y = carve(ws, P);
    if (!ws || ws_bytes < Y.bytes || !fipt_aligned(ws, 256))
        return fipt_set_error(FIPT_ERR_WORKSPACE, "voxel workspace %zu < %zu bytes (256-aligned)",
                              ws_bytes, Y.bytes);
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nv = (int64_t)R * R * R;
    FIPT_CUDA(cudaMemsetAsync(grid, 0, sizeof(float4) * (size_t)nv, st));
    if (P == 0) return FIPT_OK;
    FIPT_LAUNCH(k_vox_keys, blocks(P, 256), 256, 0, st, x, x_stride, P, s->cst, R, Y.keys, Y.vals);
    int bits = 0;
    while (((int64_t)1 << bits) < nv) ++bits;
    bits = (bits + 7) & ~7;
    uint32_t *sk, *sv;
    fipt_status r = radix_sort_pairs<uint32_t>(Y.keys, Y.keys_alt, Y.vals, Y.vals_alt, Y.hist, P,
                                               bits > 0 ? bits : 8, st, &sk, &sv);
    if (r != FIPT_OK) return r;
    const int64_t nt = (P + HEAD_TILE - 1) / HEAD_TILE;
    FIPT_LAUNCH(k_vox_count, (unsigned)nt, HEAD_TILE, 0, st, sk, P, Y.tcount);
    FIPT_LAUNCH(k_vox_scan, 1, HEAD_TILE, 0, st, Y.tcount, nt, Y.heads, Y.nhead, P);
    FIPT_LAUNCH(k_vox_compact, (unsigned)nt, HEAD_TILE, 0, st, sk, P, Y.tcount, Y.heads);
    // one run per thread at most (there are at most P runs)
    const unsigned mean_blocks = (unsigned)((P + MEAN_THREADS - 1) / MEAN_THREADS);
    FIPT_LAUNCH(k_vox_means, mean_blocks, MEAN_THREADS, 0, st, sk, sv, Y.heads, Y.nhead, L,
                reinterpret_cast<float4*>(grid));
    FIPT_LAUNCHED("voxel cache build");
    return FIPT_OK;
}

extern "C" fipt_status fipt_scene_set_voxel_cache(fipt_scene* s, const float* grid, int32_t R) {
    FIPT_REQUIRE(s, "scene is NULL");
    if (!grid) {
        s->vox = nullptr;
        s->vox_r = 0;
        return FIPT_OK;
    }
    FIPT_REQUIRE(R >= 1 && R <= 1024 && fipt_aligned(grid, 16), "bad voxel grid");
    s->vox = reinterpret_cast<const float4*>(grid);
    s->vox_r = R;
    return FIPT_OK;
}
