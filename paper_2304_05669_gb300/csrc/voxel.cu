// Voxel radiance cache (Sec. 4.2): the input pixels' radiance is
// average-pooled onto an R^3 grid spanned over the scene box and queried at
// the voxel containing a hit point (the paper uses R = 256).  Pixels are
// assigned to voxels with correctly rounded FP64 operations (as the Morton
// quantisation), grouped by a stable radix sort on the voxel index, and each
// voxel's mean is summed in pixel order in FP64, so the grid is
// deterministic.
#include "fipt_internal.cuh"

namespace {

// The per-axis scale R / (hi - lo) is the same correctly rounded double for
// every pixel; the first three threads of a block compute it once.
__global__ void k_vox_keys(const float* __restrict__ x, int64_t stride, int64_t P,
                           const SceneConst* __restrict__ c, int R, uint32_t* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
    __shared__ double scale[3];
    if (threadIdx.x < 3) {
        const double ext = __dsub_rn((double)c->hi[threadIdx.x], (double)c->lo[threadIdx.x]);
        scale[threadIdx.x] = ext > 0.0 ? __ddiv_rn((double)R, ext) : 0.0;
    }
    __syncthreads();
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    uint32_t ix[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double lo = (double)c->lo[a];
        double f = 0.0;
        if (scale[a] > 0.0) f = __dmul_rn(__dsub_rn((double)x[p * stride + a], lo), scale[a]);
        double fl = floor(f);
        fl = fl < 0.0 ? 0.0 : (fl > (double)(R - 1) ? (double)(R - 1) : fl);
        ix[a] = (uint32_t)fl;
    }
    keys[p] = (ix[2] * (uint32_t)R + ix[1]) * (uint32_t)R + ix[0];
    vals[p] = (uint32_t)p;
}

__global__ void k_vox_means(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ pix,
                            int64_t P, const float* __restrict__ L, float4* __restrict__ grid) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= P) return;
    const uint32_t k = keys[j];
    if (j > 0 && keys[j - 1] == k) return;          // not the first pixel of its voxel
    // the segment's pixels are fetched 8 at a time (independent loads in
    // flight together) and added strictly in order
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    int64_t e = j;
    bool more = true;
    while (more) {
        float v[8][3];
        bool in[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) in[u] = e + u < P && keys[e + u] == k;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (u > 0) in[u] = in[u] && in[u - 1];
            const int64_t q = in[u] ? (int64_t)pix[e + u] : 0;
            v[u][0] = in[u] ? L[3 * q] : 0.0f;
            v[u][1] = in[u] ? L[3 * q + 1] : 0.0f;
            v[u][2] = in[u] ? L[3 * q + 2] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (in[u]) {
                s0 += (double)v[u][0];
                s1 += (double)v[u][1];
                s2 += (double)v[u][2];
                ++e;
            }
        }
        more = in[7];
    }
    const double n = (double)(e - j);
    grid[k] = make_float4((float)(s0 / n), (float)(s1 / n), (float)(s2 / n), (float)n);
}

struct VoxLayout {
    uint32_t *keys, *keys_alt, *vals, *vals_alt, *hist;
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
    FIPT_LAUNCH(k_vox_means, blocks(P, 256), 256, 0, st, sk, sv, P, L, reinterpret_cast<float4*>(grid));
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
