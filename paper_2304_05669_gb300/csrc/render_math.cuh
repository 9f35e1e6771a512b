// Per-point arithmetic of the factorized render (Eq. 5 with the lerp of
// Eq. 8) and of the tone-mapped loss of Eq. 14 (alpha = 0) with its
// gradient, shared by the render kernels (render.cu) and the server's
// resident loop (trace.cu), so that a served render gives the same bits as
// fipt_render_fwd_grad.  The loss is reduced in a fixed order: a point's
// three channels and 32 consecutive points in float32 (shuffle order),
// then the RENDER_BLOCK points of a block in FP64 by warp in order
// (one partial per block), then the partials by RENDER_SUM_THREADS strided
// FP64 sums, a shuffle per warp and the warps in order.
#pragma once

#include "fipt_internal.cuh"

namespace fipt_render {

constexpr int RENDER_BLOCK = 128;        // points per loss partial (the render kernels' block)
constexpr int RENDER_SUM_THREADS = 128;  // threads of the final sum over the partials

struct Grid {
    int K;
    float s[FIPT_MAX_K];
};

struct Lerp {
    int i;
    float t;
    float inv_w;
    bool clamped;
};

__device__ __forceinline__ Lerp lerp_of(float rough, const Grid& g) {
    Lerp l;
    const float lo = g.s[0], hi = g.s[g.K - 1];
    l.clamped = rough < lo || rough > hi;
    const float s = fminf(fmaxf(rough, lo), hi);
    int i = 0;
#pragma unroll
    for (int k = 1; k < FIPT_MAX_K - 1; ++k)
        if (k <= g.K - 2 && g.s[k] <= s) i = k;
    l.i = i;
    const float w = g.s[i + 1] - g.s[i];
    l.inv_w = 1.0f / w;
    l.t = (s - g.s[i]) / w;
    return l;
}

// y^(1/2.4) for y > 0.0031308 as 2^(log2(y) / 2.4): with |log2 y| < 8.4
// the exponent is off by at most a few 1e-7, so is the power (relative).
__device__ __forceinline__ float srgb_pow(float y) { return exp2f(log2f(y) * (1.0f / 2.4f)); }

// Gamma of Eq. 14: sRGB transfer curve of y = log(1 + max(x, 0)).
__device__ __forceinline__ float tonemap(float x) {
    const float y = log1pf(fmaxf(x, 0.0f));
    return y <= 0.0031308f ? 12.92f * y : 1.055f * srgb_pow(y) - 0.055f;
}

// Gamma(x) and its derivative dt from one logarithm and one power:
// d/dx of 1.055 y^(1/2.4) is (1.055 / 2.4) y^(1/2.4) / y / (1 + x); 0 for x < 0.
__device__ __forceinline__ float tonemap_d(float x, float& dt) {
    const float y = log1pf(fmaxf(x, 0.0f));
    if (y <= 0.0031308f) {
        dt = x < 0.0f ? 0.0f : 12.92f / (1.0f + x);
        return 12.92f * y;
    }
    const float pw = srgb_pow(y);
    dt = (1.055f / 2.4f) * (pw / y) / (1.0f + x);
    return 1.055f * pw - 0.055f;
}

struct PointShade {
    float Ld[3], S0[3], S1[3], dS0[3], dS1[3];
    float a[3], m;
    Lerp l;
};

__device__ __forceinline__ void load_point(int64_t p, int K, const Grid& g, const float* Ld,
                                           const float* Ls0, const float* Ls1, const float* albedo,
                                           const float* rough, const float* metal, PointShade& P,
                                           bool with_slopes) {
    P.l = lerp_of(rough[p], g);
    const float t = P.l.t;
    const float* s0 = Ls0 + (p * K + P.l.i) * 3;
    const float* s1 = Ls1 + (p * K + P.l.i) * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        P.Ld[c] = Ld[3 * p + c];
        const float a0 = s0[c], b0 = s0[3 + c], a1 = s1[c], b1 = s1[3 + c];
        P.S0[c] = (1.0f - t) * a0 + t * b0;
        P.S1[c] = (1.0f - t) * a1 + t * b1;
        if (with_slopes) {
            P.dS0[c] = (b0 - a0) * P.l.inv_w;
            P.dS1[c] = (b1 - a1) * P.l.inv_w;
        }
        P.a[c] = albedo[3 * p + c];
    }
    P.m = metal[p];
}

// Point p's forward, loss and loss gradient (upstream gradient 1): writes
// Lr and the three gradients, returns the point's loss (float32 sum of its
// channels; 0 where the mask leaves the point out).
__device__ __forceinline__ float render_point_fwd_grad(int64_t p, const Grid& g, const float* __restrict__ Ld,
                                                       const float* __restrict__ Ls0,
                                                       const float* __restrict__ Ls1,
                                                       const float* __restrict__ albedo,
                                                       const float* __restrict__ rough,
                                                       const float* __restrict__ metal,
                                                       const float* __restrict__ Lgt,
                                                       const uint8_t* __restrict__ mask, float* __restrict__ Lr,
                                                       float* __restrict__ g_albedo, float* __restrict__ g_rough,
                                                       float* __restrict__ g_metal) {
    float loss = 0.0f;
    PointShade P;
    load_point(p, g.K, g, Ld, Ls0, Ls1, albedo, rough, metal, P, true);
    const bool on = !mask || mask[p];
    const float m = P.m;
    float gs = 0.0f, gm = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float a = P.a[c];
        const float kd = a * (1.0f - m);
        const float ks = 0.04f * (1.0f - m) + a * m;
        const float lr = kd * P.Ld[c] + ks * P.S0[c] + P.S1[c];
        Lr[3 * p + c] = lr;
        float dt;
        const float d = tonemap_d(lr, dt) - tonemap(Lgt[3 * p + c]);
        if (on) loss += d * d;
        const float gc = on ? 2.0f * d * dt : 0.0f;
        g_albedo[3 * p + c] = gc * ((1.0f - m) * P.Ld[c] + m * P.S0[c]);
        gm += gc * (-a * P.Ld[c] + (a - 0.04f) * P.S0[c]);
        gs += gc * (ks * P.dS0[c] + P.dS1[c]);
    }
    g_rough[p] = P.l.clamped ? 0.0f : gs;
    g_metal[p] = gm;
    return loss;
}

// A warp's 32 float32 losses summed down to lane 0 (shuffle order).
__device__ __forceinline__ float warp_sum_down(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_down(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace fipt_render
