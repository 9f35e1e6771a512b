// Stage-3 path-traced refinement of the shading terms (Sec. 4.3, Eq. 10),
// with multiple importance sampling (Sec. 6): a sample starts like the
// stage-1 bake (same lobe, same Philox stream), and grows its path through
// surfaces with roughness <= sigma_c by sampling the full BRDF of Eq. 1,
// until it reaches an emitter (L_e, front face only) or a rougher surface
// (the diffuse cache L').  With MIS every vertex also draws a point on the
// emitters (area-uniform) and the two strategies are combined with the
// power heuristic.
//
// Philox counters (lobe: 0 diffuse, k+1 roughness level k):
//   lobe direction at x         (pid, s, lobe, rid)                    words 0, 1
//   emitter sample at x         (pid, s, lobe | 0x100, rid)            words 0 (triangle), 1, 2 (point)
//   BRDF at path vertex i >= 1  (pid, s, lobe | i << 9, rid)           words 0, 1 (direction), 2 (lobe)
//   emitter sample at vertex i  (pid, s, lobe | i << 9 | 0x100, rid)   words 0, 1, 2
// At a vertex the diffuse lobe is drawn with probability
// P_d = clamp(mean(k_d) / (mean(k_d) + mean(k_s)), 0.1, 0.9); vertices seen
// at n.wo <= 1e-2 drop the specular lobe (P_d = 1).
#include "fipt_internal.cuh"

namespace {

constexpr int REFINE_THREADS = 128;
constexpr float PI_F = 3.14159265358979f;

struct RefineArgs {
    BakeArgs A;
    float sigma_c;
    int max_depth;
    int mis;
    int smax;               // stride of the per-sample output
};

__device__ __forceinline__ float ggx_d(float sin2, float cos2, float a2) {
    const float den = sin2 + a2 * cos2;
    return a2 / (PI_F * den * den);
}

// sin^2 of the angle between unit vectors n and h as |n x h|^2 (accurate
// near zero, where 1 - (n.h)^2 cancels).
__device__ __forceinline__ float sin2_between(float3 n, float hx, float hy, float hz) {
    const float cx = n.y * hz - n.z * hy, cy = n.z * hx - n.x * hz, cz = n.x * hy - n.y * hx;
    return cx * cx + cy * cy + cz * cz;
}

__device__ __forceinline__ float smith_g1(float mu, float a2) {
    return 2.0f * mu / (mu + sqrtf(a2 + (1.0f - a2) * mu * mu));
}

__device__ __forceinline__ float4 u4(uint32_t pid, uint32_t s, uint32_t lane, const BakeArgs& A) {
    const uint4 r = philox4x32_10(make_uint4(pid, s, lane, A.request_id), A.key);
    return make_float4(u24f(r.x), u24f(r.y), u24f(r.z), u24f(r.w));
}

__device__ __forceinline__ bool is_emitter(const float4 le) {
    return le.x > 0.0f || le.y > 0.0f || le.z > 0.0f;
}

// Point on the emitters: triangle k = first with cdf[k] > u.x * A, uniform
// point by the square-root map.  Returns the emitter's leaf.
__device__ __forceinline__ int emitter_sample(const SceneView& sc, int n_emit, double A, float4 u,
                                              float3& y) {
    const double target = (double)u.x * A;
    int lo = 0, hi = n_emit - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sc.emit_cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    const int leaf = sc.emit_leaf[lo];
    const float4 p0 = __ldg(sc.tris + 3 * leaf), p1 = __ldg(sc.tris + 3 * leaf + 1),
                 p2 = __ldg(sc.tris + 3 * leaf + 2);
    const float r1 = sqrtf(u.y);
    const float b0 = 1.0f - r1, b1 = r1 * (1.0f - u.z), b2 = r1 * u.z;
    y = make_float3(b0 * p0.x + b1 * p1.x + b2 * p2.x, b0 * p0.y + b1 * p1.y + b2 * p2.y,
                    b0 * p0.z + b1 * p1.z + b2 * p2.z);
    return leaf;
}

// Unit face normal of a leaf (not oriented) and twice its area.
__device__ __forceinline__ float3 leaf_normal(const SceneView& sc, int leaf) {
    const float4 p0 = __ldg(sc.tris + 3 * leaf), p1 = __ldg(sc.tris + 3 * leaf + 1),
                 p2 = __ldg(sc.tris + 3 * leaf + 2);
    const float e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
    const float e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float il = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
    return make_float3(nx * il, ny * il, nz * il);
}

struct Mat {
    float kd[3], ks[3];
    float a2;
    float Pd;
    bool spec;
};

__device__ __forceinline__ Mat vertex_mat(const SceneView& sc, int leaf, float mu_o) {
    const float4 m0 = __ldg(sc.mats + 2 * leaf), m1 = __ldg(sc.mats + 2 * leaf + 1);
    Mat M;
    const float m = m1.x;
    const float a[3] = {m0.x, m0.y, m0.z};
    float kd = 0.0f, ks = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        M.kd[c] = a[c] * (1.0f - m);
        M.ks[c] = 0.04f * (1.0f - m) + a[c] * m;
        kd += M.kd[c];
        ks += M.ks[c];
    }
    const float al = m0.w * m0.w;
    M.a2 = al * al;
    float Pd = kd / (kd + ks);
    Pd = fminf(fmaxf(Pd, 0.1f), 0.9f);
    M.spec = mu_o > 1e-2f;
    M.Pd = M.spec ? Pd : 1.0f;
    return M;
}

// Full BRDF of Eq. 1 (cosine included) and the vertex's mixture pdf.  When
// hs is given, wi was reflected about that sampled half vector and D is
// evaluated there (sin2h = its squared sine), not at a recomputed one.
__device__ __forceinline__ void vertex_brdf(const Mat& M, float3 n, float3 wo, float3 wi, float mu_o,
                                            float f[3], float& pdf, const float3* hs = nullptr,
                                            float sin2h = 0.0f) {
    f[0] = f[1] = f[2] = 0.0f;
    pdf = 0.0f;
    const float mu_i = n.x * wi.x + n.y * wi.y + n.z * wi.z;
    if (mu_i <= 0.0f) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = M.kd[c] * mu_i / PI_F;
    pdf = M.Pd * mu_i / PI_F;
    if (!M.spec) return;
    float hx, hy, hz;
    if (hs) {
        hx = hs->x; hy = hs->y; hz = hs->z;
    } else {
        hx = wi.x + wo.x; hy = wi.y + wo.y; hz = wi.z + wo.z;
        const float hl = 1.0f / sqrtf(hx * hx + hy * hy + hz * hz);
        hx *= hl; hy *= hl; hz *= hl;
    }
    const float ch = n.x * hx + n.y * hy + n.z * hz;
    const float co = wo.x * hx + wo.y * hy + wo.z * hz;
    if (ch <= 0.0f || co <= 0.0f) return;
    const float D = ggx_d(hs ? sin2h : sin2_between(n, hx, hy, hz), ch * ch, M.a2);
    const float G = smith_g1(mu_i, M.a2) * smith_g1(mu_o, M.a2);
    const float x1 = 1.0f - co, x2 = x1 * x1, F1 = x2 * x2 * x1, F0 = 1.0f - F1;
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] += (M.ks[c] * F0 + F1) * D * G / (4.0f * mu_o);
    pdf += (1.0f - M.Pd) * D * ch / (4.0f * co);
}

__device__ __forceinline__ float3 to_world(float3 t, float3 b, float3 n, float x, float y, float z) {
    return make_float3(x * t.x + y * b.x + z * n.x, x * t.y + y * b.y + z * n.y,
                       x * t.z + y * b.z + z * n.z);
}

// Radiance arriving along the ray (o, d) that leaves a surface point on
// original triangle skip0, estimated from its first hit on (Eq. 10 + MIS).
template <int STRIDE>
__device__ void path_radiance(const SceneView& sc, const RefineArgs& R, int n_emit, double A_emit,
                              float3 o, float3 d, int skip, float pdf_prev, uint32_t pid, uint32_t s,
                              uint32_t lobe, float L[3], int* stack, int32_t* status) {
    float beta[3] = {1.0f, 1.0f, 1.0f};
    L[0] = L[1] = L[2] = 0.0f;
    const float eps = sc.cst->eps;
    for (int depth = 1;; ++depth) {
        const TraceRay r = make_ray(o.x, o.y, o.z, d.x, d.y, d.z);
        BestHit h;
        closest_hit<STRIDE>(sc, r, skip, stack, h, status);
        if (h.leaf < 0) {
            if (sc.env) {
                const float3 e = env_lookup(sc, d.x, d.y, d.z);
                L[0] += beta[0] * e.x;
                L[1] += beta[1] * e.y;
                L[2] += beta[2] * e.z;
            }
            return;
        }
        const float4 le = __ldg(sc.shade + 2 * h.leaf);
        if (is_emitter(le)) {
            if (!h.front) return;
            float w = 1.0f;
            if (R.mis && n_emit > 0) {
                const float3 ne = leaf_normal(sc, h.leaf);
                const float ce = fabsf(d.x * ne.x + d.y * ne.y + d.z * ne.z);
                const float pl = (float)((double)h.t * h.t / (A_emit * ce));
                w = pdf_prev * pdf_prev / (pdf_prev * pdf_prev + pl * pl);
            }
            L[0] += beta[0] * w * le.x;
            L[1] += beta[1] * w * le.y;
            L[2] += beta[2] * w * le.z;
            return;
        }
        const float4 m0 = __ldg(sc.mats + 2 * h.leaf);
        if (m0.w > R.sigma_c) {
            float3 ca;
            if (sc.vox) {
                ca = voxel_lookup(sc, o.x + h.t * d.x, o.y + h.t * d.y, o.z + h.t * d.z);
            } else {
                const float4 c4 = __ldg(sc.shade + 2 * h.leaf + 1);
                ca = make_float3(c4.x, c4.y, c4.z);
            }
            L[0] += beta[0] * ca.x;
            L[1] += beta[1] * ca.y;
            L[2] += beta[2] * ca.z;
            return;
        }
        if (depth > R.max_depth) return;
        // a smooth surface: continue the path
        float3 n = leaf_normal(sc, h.leaf);
        const float3 wo = make_float3(-d.x, -d.y, -d.z);
        if (n.x * wo.x + n.y * wo.y + n.z * wo.z < 0.0f) n = make_float3(-n.x, -n.y, -n.z);
        const float3 x = make_float3(o.x + h.t * d.x, o.y + h.t * d.y, o.z + h.t * d.z);
        const float3 xo = make_float3(x.x + eps * n.x, x.y + eps * n.y, x.z + eps * n.z);
        const float mu_o = n.x * wo.x + n.y * wo.y + n.z * wo.z;
        const Mat M = vertex_mat(sc, h.leaf, mu_o);
        const uint32_t lane = lobe | ((uint32_t)depth << 9);
        if (R.mis && n_emit > 0) {
            float3 y;
            const int e = emitter_sample(sc, n_emit, A_emit, u4(pid, s, lane | 0x100u, R.A), y);
            float wx = y.x - xo.x, wy = y.y - xo.y, wz = y.z - xo.z;
            const float dist = sqrtf(wx * wx + wy * wy + wz * wz);
            wx /= dist; wy /= dist; wz /= dist;
            const float3 ne = leaf_normal(sc, e);
            const float ce = -(wx * ne.x + wy * ne.y + wz * ne.z);
            if (ce > 0.0f) {
                float f[3], pb;
                vertex_brdf(M, n, wo, make_float3(wx, wy, wz), mu_o, f, pb);
                if (f[0] > 0.0f || f[1] > 0.0f || f[2] > 0.0f) {
                    BestHit vh;
                    closest_hit<STRIDE>(sc, make_ray(xo.x, xo.y, xo.z, wx, wy, wz), h.orig, stack, vh,
                                        status);
                    if (vh.leaf == e) {
                        const float pl = (float)((double)dist * dist / (A_emit * ce));
                        const float w = pl * pl / (pl * pl + pb * pb);
                        const float4 lee = __ldg(sc.shade + 2 * e);
                        L[0] += beta[0] * w * lee.x * f[0] / pl;
                        L[1] += beta[1] * w * lee.y * f[1] / pl;
                        L[2] += beta[2] * w * lee.z * f[2] / pl;
                    }
                }
            }
        }
        const float4 u = u4(pid, s, lane, R.A);
        float3 tb, bb;
        onb(n.x, n.y, n.z, tb, bb);
        float3 wi, hh = make_float3(0.0f, 0.0f, 1.0f);
        float sin2h = 0.0f;
        float sn, cs;
        sincospif(2.0f * u.y, &sn, &cs);
        const bool glossy = !(u.z < M.Pd);
        if (!glossy) {
            const float rr = sqrtf(u.x);
            wi = to_world(tb, bb, n, rr * cs, rr * sn, sqrtf(1.0f - u.x));
        } else {
            const float om = 1.0f - u.x;
            const float den = om + M.a2 * u.x;
            sin2h = M.a2 * u.x / den;
            const float ch = sqrtf(om / den), sh = sqrtf(sin2h);
            hh = to_world(tb, bb, n, sh * cs, sh * sn, ch);
            const float c = wo.x * hh.x + wo.y * hh.y + wo.z * hh.z;
            wi = make_float3(2.0f * c * hh.x - wo.x, 2.0f * c * hh.y - wo.y, 2.0f * c * hh.z - wo.z);
        }
        float f[3], pdf;
        vertex_brdf(M, n, wo, wi, mu_o, f, pdf, glossy ? &hh : nullptr, sin2h);
        if (pdf <= 0.0f) return;
        beta[0] *= f[0] / pdf;
        beta[1] *= f[1] / pdf;
        beta[2] *= f[2] / pdf;
        o = xo;
        d = wi;
        skip = h.orig;
        pdf_prev = pdf;
    }
}

template <bool PER_SAMPLE>
__global__ void __launch_bounds__(REFINE_THREADS)
k_refine(SceneView sc, const fipt_query* __restrict__ q, int64_t N, RefineArgs R, float* __restrict__ Ld,
         float* __restrict__ Ls0, float* __restrict__ Ls1, float* __restrict__ per_sample,
         int32_t* status) {
    __shared__ int stk[STACK_DEPTH * REFINE_THREADS];
    int* stack = stk + threadIdx.x;
    const BakeArgs& A = R.A;
    const int K = A.K, L = 1 + K;
    const int64_t g = blockIdx.x * (int64_t)REFINE_THREADS + threadIdx.x;
    const int64_t w = g >> 5;
    const int lane = (int)(g & 31);
    const int lobe = (int)(w % L);
    const int64_t p = (w / L) * 32 + lane;
    if (p >= N) return;
    const float2* qp = reinterpret_cast<const float2*>(q + p);
    const float2 q0 = qp[0], q1 = qp[1], q2 = qp[2], q3 = qp[3], q4 = qp[4];
    float3 n = make_float3(q1.y, q2.x, q2.y);
    float3 wo = make_float3(q3.x, q3.y, q4.x);
    const int skip = __float_as_int(q4.y);
    {
        const float il = 1.0f / sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
        n = make_float3(n.x * il, n.y * il, n.z * il);
        const float jl = 1.0f / sqrtf(wo.x * wo.x + wo.y * wo.y + wo.z * wo.z);
        wo = make_float3(wo.x * jl, wo.y * jl, wo.z * jl);
    }
    const float mu_o = n.x * wo.x + n.y * wo.y + n.z * wo.z;
    const int S = lobe == 0 ? A.spp_d : A.spp_s;
    float* ps = PER_SAMPLE ? per_sample + ((size_t)(p * L + lobe) * R.smax) * 6 : nullptr;
    if (lobe > 0 && mu_o <= 1e-2f) {
        float* o0 = Ls0 + (p * K + (lobe - 1)) * 3;
        float* o1 = Ls1 + (p * K + (lobe - 1)) * 3;
        o0[0] = o0[1] = o0[2] = 0.0f;
        o1[0] = o1[1] = o1[2] = 0.0f;
        if (PER_SAMPLE)
            for (int s = 0; s < R.smax * 6; ++s) ps[s] = 0.0f;
        return;
    }
    float a2 = 0.0f, g1o = 0.0f;
    if (lobe > 0) {
        float sg = A.sigma[0];
#pragma unroll
        for (int k = 1; k < FIPT_MAX_K; ++k)
            if (lobe - 1 == k) sg = A.sigma[k];
        const float al = sg * sg;
        a2 = al * al;
        g1o = smith_g1(mu_o, a2);
    }
    float3 tb, bb;
    onb(n.x, n.y, n.z, tb, bb);
    const float eps = sc.cst->eps;
    const float3 o = make_float3(q0.x + eps * n.x, q0.y + eps * n.y, q1.x + eps * n.z);
    const uint32_t pid = A.point_base + (uint32_t)p;
    const int n_emit = sc.cst->n_emit;
    const double A_emit = sc.cst->A_emit;
    float acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < S; ++s) {
        float c6[6] = {0, 0, 0, 0, 0, 0};
        if (R.mis && n_emit > 0) {            // emitter sample at x
            float3 y;
            const int e = emitter_sample(sc, n_emit, A_emit, u4(pid, (uint32_t)s, (uint32_t)lobe | 0x100u, A), y);
            float wx = y.x - o.x, wy = y.y - o.y, wz = y.z - o.z;
            const float dist = sqrtf(wx * wx + wy * wy + wz * wz);
            wx /= dist; wy /= dist; wz /= dist;
            const float3 ne = leaf_normal(sc, e);
            const float ce = -(wx * ne.x + wy * ne.y + wz * ne.z);
            const float mu_i = n.x * wx + n.y * wy + n.z * wz;
            float g0 = 0.0f, g1 = 0.0f, pb = 0.0f;
            if (ce > 0.0f && mu_i > 0.0f) {
                if (lobe == 0) {
                    g0 = mu_i / PI_F;
                    pb = g0;
                } else {
                    float hx = wx + wo.x, hy = wy + wo.y, hz = wz + wo.z;
                    const float hl = 1.0f / sqrtf(hx * hx + hy * hy + hz * hz);
                    hx *= hl; hy *= hl; hz *= hl;
                    const float ch = n.x * hx + n.y * hy + n.z * hz;
                    const float c = wo.x * hx + wo.y * hy + wo.z * hz;
                    if (ch > 0.0f && c > 0.0f) {
                        const float D = ggx_d(sin2_between(n, hx, hy, hz), ch * ch, a2);
                        const float G = smith_g1(mu_i, a2) * g1o;
                        const float x1 = 1.0f - c, x2 = x1 * x1, F1 = x2 * x2 * x1;
                        g0 = (1.0f - F1) * D * G / (4.0f * mu_o);
                        g1 = F1 * D * G / (4.0f * mu_o);
                        pb = D * ch / (4.0f * c);
                    }
                }
            }
            if (g0 > 0.0f || g1 > 0.0f) {
                BestHit vh;
                closest_hit<REFINE_THREADS>(sc, make_ray(o.x, o.y, o.z, wx, wy, wz), skip, stack, vh,
                                            status);
                if (vh.leaf == e) {
                    const float pl = (float)((double)dist * dist / (A_emit * ce));
                    const float wgt = pl * pl / (pl * pl + pb * pb);
                    const float4 lee = __ldg(sc.shade + 2 * e);
                    c6[0] += wgt * lee.x * g0 / pl; c6[1] += wgt * lee.y * g0 / pl; c6[2] += wgt * lee.z * g0 / pl;
                    c6[3] += wgt * lee.x * g1 / pl; c6[4] += wgt * lee.y * g1 / pl; c6[5] += wgt * lee.z * g1 / pl;
                }
            }
        }
        // lobe sample at x (the stage-1 sampler)
        const float4 u = u4(pid, (uint32_t)s, (uint32_t)lobe, A);
        float sn, cs;
        sincospif(2.0f * u.y, &sn, &cs);
        float3 wi;
        float W0 = 1.0f, W1 = 0.0f, pb = 0.0f;
        bool valid = true;
        if (lobe == 0) {
            const float rr = sqrtf(u.x), lz = sqrtf(1.0f - u.x);
            wi = to_world(tb, bb, n, rr * cs, rr * sn, lz);
            pb = lz / PI_F;
        } else {
            const float om = 1.0f - u.x;
            const float den = om + a2 * u.x;
            const float cos2 = om / den, sin2 = a2 * u.x / den;
            const float ch = sqrtf(cos2), sh = sqrtf(sin2);
            const float3 h = to_world(tb, bb, n, sh * cs, sh * sn, ch);
            const float c = wo.x * h.x + wo.y * h.y + wo.z * h.z;
            wi = make_float3(2.0f * c * h.x - wo.x, 2.0f * c * h.y - wo.y, 2.0f * c * h.z - wo.z);
            const float mu_i = n.x * wi.x + n.y * wi.y + n.z * wi.z;
            if (mu_i <= 0.0f || c <= 0.0f) {
                valid = false;
            } else {
                const float wt = smith_g1(mu_i, a2) * g1o * c / (mu_o * ch);
                const float x1 = 1.0f - c, x2 = x1 * x1, F1 = x2 * x2 * x1;
                W0 = (1.0f - F1) * wt;
                W1 = F1 * wt;
                pb = ggx_d(sin2, cos2, a2) * ch / (4.0f * c);
            }
        }
        if (valid) {
            float Lp[3];
            path_radiance<REFINE_THREADS>(sc, R, n_emit, A_emit, o, wi, skip, pb, pid, (uint32_t)s,
                                          (uint32_t)lobe, Lp, stack, status);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                c6[c] += W0 * Lp[c];
                c6[3 + c] += W1 * Lp[c];
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i] += c6[i];
        if (PER_SAMPLE)
            for (int i = 0; i < 6; ++i) ps[s * 6 + i] = c6[i];
    }
    if (PER_SAMPLE)
        for (int s = S; s < R.smax; ++s)
            for (int i = 0; i < 6; ++i) ps[s * 6 + i] = 0.0f;
    const float fs = (float)S;
    if (lobe == 0) {
        Ld[3 * p + 0] = acc[0] / fs;
        Ld[3 * p + 1] = acc[1] / fs;
        Ld[3 * p + 2] = acc[2] / fs;
    } else {
        float* o0 = Ls0 + (p * K + (lobe - 1)) * 3;
        float* o1 = Ls1 + (p * K + (lobe - 1)) * 3;
        o0[0] = acc[0] / fs; o0[1] = acc[1] / fs; o0[2] = acc[2] / fs;
        o1[0] = acc[3] / fs; o1[1] = acc[4] / fs; o1[2] = acc[5] / fs;
    }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" fipt_status fipt_bake_refine(fipt_scene* s, const fipt_query* q, int64_t N,
                                        const fipt_bake_params* prm, float sigma_c, int32_t max_depth,
                                        int32_t mis, float* Ld, float* Ls0, float* Ls1,
                                        float* per_sample, fipt_stream stream) {
    FIPT_REQUIRE(s && prm, "scene / params is NULL");
    FIPT_REQUIRE(s->has_materials, "fipt_scene_set_materials must be called before a refinement");
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 32), "bad point count %lld", (long long)N);
    FIPT_REQUIRE(prm->K >= 1 && prm->K <= FIPT_MAX_K, "K must be in [1, %d]", FIPT_MAX_K);
    FIPT_REQUIRE(prm->spp_diffuse >= 1 && prm->spp_specular >= 1, "spp must be >= 1");
    FIPT_REQUIRE(max_depth >= 0 && max_depth < 4096, "max_depth must be in [0, 4096)");
    for (int k = 0; k < prm->K; ++k)
        FIPT_REQUIRE(prm->sigma[k] > 0.0f && prm->sigma[k] <= 1.0f, "sigma[%d] not in (0, 1]", k);
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(q && Ld && Ls0 && Ls1, "NULL query / output array");
    FIPT_REQUIRE(fipt_aligned(q, 8) && fipt_aligned(Ld, 4) && fipt_aligned(Ls0, 4) &&
                 fipt_aligned(Ls1, 4) && fipt_aligned(per_sample, 4), "misaligned array");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    RefineArgs R;
    R.A.key = make_uint2((uint32_t)prm->seed, (uint32_t)(prm->seed >> 32));
    R.A.request_id = prm->request_id;
    R.A.point_base = prm->point_base;
    R.A.spp_d = prm->spp_diffuse;
    R.A.spp_s = prm->spp_specular;
    R.A.K = prm->K;
    for (int k = 0; k < FIPT_MAX_K; ++k) R.A.sigma[k] = k < prm->K ? prm->sigma[k] : 1.0f;
    R.sigma_c = sigma_c;
    R.max_depth = max_depth;
    R.mis = mis != 0;
    R.smax = prm->spp_diffuse > prm->spp_specular ? prm->spp_diffuse : prm->spp_specular;
    const int64_t threads = ((N + 31) / 32) * (1 + prm->K) * 32;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (per_sample)
        FIPT_LAUNCH(k_refine<true>, blocks(threads, REFINE_THREADS), REFINE_THREADS, 0, st, s->view(), q,
                    N, R, Ld, Ls0, Ls1, per_sample, s->ctx->status);
    else
        FIPT_LAUNCH(k_refine<false>, blocks(threads, REFINE_THREADS), REFINE_THREADS, 0, st, s->view(),
                    q, N, R, Ld, Ls0, Ls1, nullptr, s->ctx->status);
    FIPT_LAUNCHED("bake_refine");
    return FIPT_OK;
}
