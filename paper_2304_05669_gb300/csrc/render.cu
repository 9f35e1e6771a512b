// Factorized render (Eq. 5 with the lerp of Eq. 8), the tone-mapped loss of
// Eq. 14 (alpha = 0) and its gradient with respect to per-point albedo,
// roughness and metallic.  The kernels stream one point per thread; the
// loss is reduced in a fixed order (per-block FP64 partials, then one block
// over the partials) so it is bit-reproducible.  k_render_fwd_grad computes
// the forward, the loss and the gradient (for an upstream gradient of 1)
// in one pass, so that a training step reads its inputs once;
// k_render_grad_scale applies the upstream gradient afterwards.
#include <algorithm>
#include <mutex>

#include "fipt_internal.cuh"
#include "render_math.cuh"

namespace {

using namespace fipt_render;
constexpr int RENDER_THREADS = RENDER_BLOCK;   // one loss partial per block

// The block's loss to partial[blockIdx.x]: a point's three channels and a
// warp's 32 points are summed in float32 (fixed shuffle order), the
// block's warps in FP64 in order.  Every thread of the block calls it.
__device__ __forceinline__ void block_loss(float loss, double* partial) {
    loss = warp_sum_down(loss);
    __shared__ double ws[RENDER_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < RENDER_THREADS / 32; ++w) s += ws[w];
        partial[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(RENDER_THREADS)
k_render_fwd(const float* __restrict__ Ld, const float* __restrict__ Ls0, const float* __restrict__ Ls1,
             int64_t N, Grid g, const float* __restrict__ albedo, const float* __restrict__ rough,
             const float* __restrict__ metal, const float* __restrict__ Lgt,
             const uint8_t* __restrict__ mask, float* __restrict__ Lr, double* __restrict__ partial) {
    const int64_t p = blockIdx.x * (int64_t)RENDER_THREADS + threadIdx.x;
    float loss = 0.0f;
    if (p < N) {
        PointShade P;
        load_point(p, g.K, g, Ld, Ls0, Ls1, albedo, rough, metal, P, false);
        const float m = P.m;
        float lr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float kd = P.a[c] * (1.0f - m);
            const float ks = 0.04f * (1.0f - m) + P.a[c] * m;
            lr[c] = kd * P.Ld[c] + ks * P.S0[c] + P.S1[c];
            Lr[3 * p + c] = lr[c];
        }
        if (Lgt && (!mask || mask[p])) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = tonemap(lr[c]) - tonemap(Lgt[3 * p + c]);
                loss += d * d;
            }
        }
    }
    if (partial) block_loss(loss, partial);
}

// One block of SUM_THREADS sums the per-block partials in a fixed order.
constexpr int SUM_THREADS = RENDER_SUM_THREADS;
__global__ void __launch_bounds__(SUM_THREADS) k_sum_partials(const double* __restrict__ partial, int64_t n,
                                                             double* __restrict__ out) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += SUM_THREADS) s += partial[i];
    s = warp_sum_down(s);
    __shared__ double ws[SUM_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < SUM_THREADS / 32; ++w) t += ws[w];
        *out = t;
    }
}

__global__ void __launch_bounds__(RENDER_THREADS)
k_render_bwd(const float* __restrict__ Ld, const float* __restrict__ Ls0, const float* __restrict__ Ls1,
             int64_t N, Grid g, const float* __restrict__ albedo, const float* __restrict__ rough,
             const float* __restrict__ metal, const float* __restrict__ Lgt,
             const uint8_t* __restrict__ mask, const double* __restrict__ grad_loss,
             float* __restrict__ g_albedo, float* __restrict__ g_rough, float* __restrict__ g_metal) {
    const int64_t p = blockIdx.x * (int64_t)RENDER_THREADS + threadIdx.x;
    if (p >= N) return;
    PointShade P;
    load_point(p, g.K, g, Ld, Ls0, Ls1, albedo, rough, metal, P, true);
    const float scale = grad_loss ? (float)*grad_loss : 1.0f;
    const bool on = !mask || mask[p];
    const float m = P.m;
    float gs = 0.0f, gm = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = P.a[c];
        const float kd = a * (1.0f - m);
        const float ks = 0.04f * (1.0f - m) + a * m;
        const float lr = kd * P.Ld[c] + ks * P.S0[c] + P.S1[c];
        float dt;
        const float d = tonemap_d(lr, dt) - tonemap(Lgt[3 * p + c]);
        const float gc = on ? 2.0f * d * dt * scale : 0.0f;
        g_albedo[3 * p + c] = gc * ((1.0f - m) * P.Ld[c] + m * P.S0[c]);
        gm += gc * (-a * P.Ld[c] + (a - 0.04f) * P.S0[c]);
        gs += gc * (ks * P.dS0[c] + P.dS1[c]);
    }
    g_rough[p] = P.l.clamped ? 0.0f : gs;
    g_metal[p] = gm;
}

// Forward, loss and loss gradient in one pass: the values of k_render_fwd
// and of k_render_bwd with grad_loss = 1, each input read once.
__global__ void __launch_bounds__(RENDER_THREADS)
k_render_fwd_grad(const float* __restrict__ Ld, const float* __restrict__ Ls0, const float* __restrict__ Ls1,
                  int64_t N, Grid g, const float* __restrict__ albedo, const float* __restrict__ rough,
                  const float* __restrict__ metal, const float* __restrict__ Lgt,
                  const uint8_t* __restrict__ mask, float* __restrict__ Lr, double* __restrict__ partial,
                  float* __restrict__ g_albedo, float* __restrict__ g_rough, float* __restrict__ g_metal) {
    const int64_t p = blockIdx.x * (int64_t)RENDER_THREADS + threadIdx.x;
    float loss = 0.0f;
    if (p < N)
        loss = render_point_fwd_grad(p, g, Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask, Lr, g_albedo, g_rough,
                                     g_metal);
    block_loss(loss, partial);
}

// Multiplies the gradients of k_render_fwd_grad by the upstream gradient
// of the loss; a factor of exactly 1 leaves them as they are.
__global__ void __launch_bounds__(RENDER_THREADS)
k_render_grad_scale(int64_t N, const double* __restrict__ grad_loss, float* __restrict__ g_albedo,
                    float* __restrict__ g_rough, float* __restrict__ g_metal) {
    const float s = (float)*grad_loss;
    if (s == 1.0f) return;
    for (int64_t p = blockIdx.x * (int64_t)RENDER_THREADS + threadIdx.x; p < N;
         p += (int64_t)gridDim.x * RENDER_THREADS) {
        g_albedo[3 * p + 0] *= s;
        g_albedo[3 * p + 1] *= s;
        g_albedo[3 * p + 2] *= s;
        g_rough[p] *= s;
        g_metal[p] *= s;
    }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

fipt_status make_grid(int32_t K, const float* sigma_grid, Grid& g) {
    FIPT_REQUIRE(K >= 2 && K <= FIPT_MAX_K, "K must be in [2, %d]", FIPT_MAX_K);
    FIPT_REQUIRE(sigma_grid, "sigma_grid (host) is NULL");
    g.K = K;
    for (int k = 0; k < FIPT_MAX_K; ++k) g.s[k] = k < K ? sigma_grid[k] : sigma_grid[K - 1];
    for (int k = 1; k < K; ++k)
        FIPT_REQUIRE(g.s[k] > g.s[k - 1], "sigma_grid must increase strictly");
    return FIPT_OK;
}

fipt_status check_render_arrays(int64_t N, const float* Ld, const float* Ls0, const float* Ls1,
                                const float* albedo, const float* rough, const float* metal) {
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 40), "bad point count");
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(Ld && Ls0 && Ls1 && albedo && rough && metal, "NULL input array");
    FIPT_REQUIRE(fipt_aligned(Ld, 4) && fipt_aligned(Ls0, 4) && fipt_aligned(Ls1, 4) &&
                 fipt_aligned(albedo, 4) && fipt_aligned(rough, 4) && fipt_aligned(metal, 4),
                 "inputs must be 4-byte aligned");
    return FIPT_OK;
}

}  // namespace

extern "C" fipt_status fipt_render_workspace_size(int64_t N, size_t* bytes) {
    FIPT_REQUIRE(bytes && N >= 0, "bad arguments");
    *bytes = (size_t)(blocks(N, RENDER_THREADS) + 1) * sizeof(double) + 256;
    return FIPT_OK;
}

extern "C" fipt_status fipt_render_fwd(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                                       int32_t K, const float* sigma_grid, const float* albedo,
                                       const float* rough, const float* metal, const float* Lgt,
                                       const uint8_t* mask, float* Lr, double* loss, void* ws,
                                       size_t ws_bytes, fipt_stream stream) {
    Grid g;
    fipt_status r = make_grid(K, sigma_grid, g);
    if (r != FIPT_OK) return r;
    r = check_render_arrays(N, Ld, Ls0, Ls1, albedo, rough, metal);
    if (r != FIPT_OK) return r;
    FIPT_REQUIRE(!Lgt || loss, "loss must be given with Lgt");
    FIPT_REQUIRE(fipt_aligned(loss, 8) && fipt_aligned(Lgt, 4) && fipt_aligned(Lr, 4),
                 "misaligned output");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (N == 0) {
        if (loss) FIPT_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
        return FIPT_OK;
    }
    FIPT_REQUIRE(Lr, "Lr is NULL");
    double* partial = nullptr;
    if (Lgt) {
        size_t need;
        fipt_render_workspace_size(N, &need);
        if (!ws || ws_bytes < need)
            return fipt_set_error(FIPT_ERR_WORKSPACE, "render workspace %zu < %zu", ws_bytes, need);
        FIPT_REQUIRE(fipt_aligned(ws, 8), "workspace must be 8-byte aligned");
        partial = static_cast<double*>(ws);
    }
    const unsigned nb = blocks(N, RENDER_THREADS);
    FIPT_LAUNCH(k_render_fwd, nb, RENDER_THREADS, 0, st, Ld, Ls0, Ls1, N, g, albedo, rough, metal, Lgt, mask,
                                                Lr, partial);
    if (Lgt) FIPT_LAUNCH(k_sum_partials, 1, SUM_THREADS, 0, st, partial, nb, loss);
    FIPT_LAUNCHED("render_fwd");
    return FIPT_OK;
}

extern "C" fipt_status fipt_render_bwd(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                                       int32_t K, const float* sigma_grid, const float* albedo,
                                       const float* rough, const float* metal, const float* Lgt,
                                       const uint8_t* mask, const double* grad_loss, float* g_albedo,
                                       float* g_rough, float* g_metal, fipt_stream stream) {
    Grid g;
    fipt_status r = make_grid(K, sigma_grid, g);
    if (r != FIPT_OK) return r;
    r = check_render_arrays(N, Ld, Ls0, Ls1, albedo, rough, metal);
    if (r != FIPT_OK) return r;
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(Lgt && g_albedo && g_rough && g_metal, "Lgt / gradient output is NULL");
    FIPT_REQUIRE(fipt_aligned(Lgt, 4) && fipt_aligned(g_albedo, 4) && fipt_aligned(g_rough, 4) &&
                 fipt_aligned(g_metal, 4) && fipt_aligned(grad_loss, 8), "misaligned array");
    FIPT_LAUNCH(k_render_bwd, blocks(N, RENDER_THREADS), RENDER_THREADS, 0, static_cast<cudaStream_t>(stream), Ld, Ls0, Ls1, N, g, albedo, rough, metal, Lgt, mask, grad_loss, g_albedo, g_rough, g_metal);
    FIPT_LAUNCHED("render_bwd");
    return FIPT_OK;
}

extern "C" fipt_status fipt_render_fwd_grad(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                                            int32_t K, const float* sigma_grid, const float* albedo,
                                            const float* rough, const float* metal, const float* Lgt,
                                            const uint8_t* mask, float* Lr, double* loss, float* g_albedo,
                                            float* g_rough, float* g_metal, void* ws, size_t ws_bytes,
                                            fipt_stream stream) {
    Grid g;
    fipt_status r = make_grid(K, sigma_grid, g);
    if (r != FIPT_OK) return r;
    r = check_render_arrays(N, Ld, Ls0, Ls1, albedo, rough, metal);
    if (r != FIPT_OK) return r;
    FIPT_REQUIRE(loss && fipt_aligned(loss, 8), "loss is NULL or misaligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (N == 0) {
        FIPT_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
        return FIPT_OK;
    }
    FIPT_REQUIRE(Lgt && Lr && g_albedo && g_rough && g_metal, "Lgt / Lr / gradient output is NULL");
    FIPT_REQUIRE(fipt_aligned(Lgt, 4) && fipt_aligned(Lr, 4) && fipt_aligned(g_albedo, 4) &&
                 fipt_aligned(g_rough, 4) && fipt_aligned(g_metal, 4), "misaligned array");
    size_t need;
    fipt_render_workspace_size(N, &need);
    if (!ws || ws_bytes < need)
        return fipt_set_error(FIPT_ERR_WORKSPACE, "render workspace %zu < %zu", ws_bytes, need);
    FIPT_REQUIRE(fipt_aligned(ws, 8), "workspace must be 8-byte aligned");
    double* partial = static_cast<double*>(ws);
    const unsigned nb = blocks(N, RENDER_THREADS);
    FIPT_LAUNCH(k_render_fwd_grad, nb, RENDER_THREADS, 0, st, Ld, Ls0, Ls1, N, g, albedo, rough, metal, Lgt,
                mask, Lr, partial, g_albedo, g_rough, g_metal);
    FIPT_LAUNCH(k_sum_partials, 1, SUM_THREADS, 0, st, partial, nb, loss);
    FIPT_LAUNCHED("render_fwd_grad");
    return FIPT_OK;
}

extern "C" fipt_status fipt_render_grad_scale(int64_t N, const double* grad_loss, float* g_albedo,
                                              float* g_rough, float* g_metal, fipt_stream stream) {
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 40), "bad point count");
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(grad_loss && g_albedo && g_rough && g_metal, "NULL argument");
    FIPT_REQUIRE(fipt_aligned(grad_loss, 8) && fipt_aligned(g_albedo, 4) && fipt_aligned(g_rough, 4) &&
                 fipt_aligned(g_metal, 4), "misaligned array");
    int dev = 0, sms = 0;
    FIPT_CUDA(cudaGetDevice(&dev));
    FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned nb = blocks(N, RENDER_THREADS);
    const unsigned grid = nb < (unsigned)(8 * sms) ? nb : (unsigned)(8 * sms);
    FIPT_LAUNCH(k_render_grad_scale, grid, RENDER_THREADS, 0, static_cast<cudaStream_t>(stream), N, grad_loss,
                g_albedo, g_rough, g_metal);
    FIPT_LAUNCHED("render_grad_scale");
    return FIPT_OK;
}

// ---------------------------------------------------------------- no-allocation variant
// Some callers cannot allocate device memory at the point where they render:
// callers whose memory comes from a fixed pool sized at start-up (embedded or
// real-time services), or threads that must not take the allocator's lock.
// fipt_render_fwd needs a caller workspace for its loss partial sums; this
// variant keeps them in a fixed array compiled into the library instead.
// The array lives on every GPU that loads the library until the process
// exits (FIPT_NOALLOC_RENDER_MAX_BLOCKS doubles = 1 MiB).
static __device__ __align__(256) double g_noalloc_partials[FIPT_NOALLOC_RENDER_MAX_BLOCKS];

namespace {
constexpr int kMaxDevices = 64;
double* g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

// Device address of g_noalloc_partials on the current device (host code
// only ever sees a host-side stand-in for the symbol).  Looked up on a
// device's first call and kept; a kept address that the driver no longer
// knows as memory of this device (the device was reset and its module
// reloaded elsewhere) is looked up again.
fipt_status noalloc_partials(double** out) {
    int dev = -1;
    FIPT_CUDA(cudaGetDevice(&dev));
    FIPT_REQUIRE(dev >= 0 && dev < kMaxDevices, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev]) {
        cudaPointerAttributes at;
        const cudaError_t e = cudaPointerGetAttributes(&at, g_noalloc_ptr[dev]);
        if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != dev) {
            (void)cudaGetLastError();      // the query's error is not the caller's
            g_noalloc_ptr[dev] = nullptr;
        }
    }
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        FIPT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return FIPT_OK;
}
}  // namespace

extern "C" fipt_status fipt_render_fwd_noalloc(const float* Ld, const float* Ls0, const float* Ls1,
                                               int64_t N, int32_t K, const float* sigma_grid,
                                               const float* albedo, const float* rough,
                                               const float* metal, const float* Lgt,
                                               const uint8_t* mask, float* Lr, double* loss,
                                               fipt_stream stream) {
    Grid g;
    fipt_status r = make_grid(K, sigma_grid, g);
    if (r != FIPT_OK) return r;
    r = check_render_arrays(N, Ld, Ls0, Ls1, albedo, rough, metal);
    if (r != FIPT_OK) return r;
    FIPT_REQUIRE(!Lgt || loss, "loss must be given with Lgt");
    FIPT_REQUIRE(fipt_aligned(loss, 8) && fipt_aligned(Lgt, 4) && fipt_aligned(Lr, 4),
                 "misaligned output");
    const int64_t nb = (N + RENDER_THREADS - 1) / RENDER_THREADS;
    if (nb > FIPT_NOALLOC_RENDER_MAX_BLOCKS)
        return fipt_set_error(FIPT_ERR_INVALID_ARG,
                              "fipt_render_fwd_noalloc: N = %lld exceeds its fixed scratch "
                              "(at most %lld points); use fipt_render_fwd with a workspace",
                              (long long)N, (long long)FIPT_NOALLOC_RENDER_MAX_BLOCKS * RENDER_THREADS);
    double* partial = nullptr;
    r = noalloc_partials(&partial);
    if (r != FIPT_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (N == 0) {
        if (loss) FIPT_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
        return FIPT_OK;
    }
    FIPT_REQUIRE(Lr, "Lr is NULL");
    // Every block writes its own partial before k_sum_partials reads exactly
    // nb of them, so nothing left over from an earlier call is ever read.
    FIPT_LAUNCH(k_render_fwd, (unsigned)nb, RENDER_THREADS, 0, st, Ld, Ls0, Ls1, N, g, albedo, rough,
                metal, Lgt, mask, Lr, Lgt ? partial : nullptr);
    if (Lgt) FIPT_LAUNCH(k_sum_partials, 1, SUM_THREADS, 0, st, partial, nb, loss);
    FIPT_LAUNCHED("render_fwd_noalloc");
    return FIPT_OK;
}
