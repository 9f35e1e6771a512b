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

#ifndef FIPT_REFINE_THREADS
#define FIPT_REFINE_THREADS 64   // small blocks: the shared stack bounds residency
#endif
#ifndef FIPT_REFINE_MINB
#define FIPT_REFINE_MINB 20      // resident blocks per SM the register budget must allow
#endif
constexpr int REFINE_THREADS = FIPT_REFINE_THREADS;
constexpr int REFINE_MINB = FIPT_REFINE_MINB;
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
                                            float f[3], float& pdf, bool use_h = false,
                                            float3 hs = make_float3(0.0f, 0.0f, 1.0f),
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
    if (use_h) {
        hx = hs.x; hy = hs.y; hz = hs.z;
    } else {
        hx = wi.x + wo.x; hy = wi.y + wo.y; hz = wi.z + wo.z;
        const float hl = 1.0f / sqrtf(hx * hx + hy * hy + hz * hz);
        hx *= hl; hy *= hl; hz *= hl;
    }
    const float ch = n.x * hx + n.y * hy + n.z * hz;
    const float co = wo.x * hx + wo.y * hy + wo.z * hz;
    if (ch <= 0.0f || co <= 0.0f) return;
    const float D = ggx_d(use_h ? sin2h : sin2_between(n, hx, hy, hz), ch * ch, M.a2);
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

// Lane state machine of the refinement.  A lane owns one (point, lobe) pair
// and walks its samples in order; each sample traces, one ray at a time:
//   K_S0   the shadow ray of the emitter sample at x (MIS only),
//   K_PATH a path segment (the lobe sample at x, then BRDF samples),
//   K_SV   the shadow ray of the emitter sample at a path vertex; the
//          vertex's BRDF sample (the next K_PATH) is drawn after it.
// All rays go through the single traversal loop of k_refine, so lanes in
// different states still walk the BVH together; a lane whose ray finished
// waits until FIPT_REFINE_REFILL lanes (or all busy lanes) are waiting, and
// the waiting lanes then consume their hits and set up their next rays
// together, as the stage-1 bake does.  Shadow rays stop looking beyond the
// sampled emitter point (only whether that emitter is the closest hit
// matters).
enum : int { K_NONE = 0, K_S0 = 1, K_PATH = 2, K_SV = 3 };
enum : int { A_START, A_MAIN, A_VERTEX_BSDF, A_END_PATH, A_END_SAMPLE, A_RAY };

#ifndef FIPT_REFINE_REFILL
#define FIPT_REFINE_REFILL 24    // lanes that must be waiting before a warp sets up new rays
#endif

__device__ __forceinline__ void start_ray(TraceRay& r, BestHit& best, int& node, int& sp, int& steps,
                                          const SceneView& sc, float ox, float oy, float oz, float dx,
                                          float dy, float dz, float tmax) {
    r = make_ray(ox, oy, oz, dx, dy, dz);
    best.t = tmax;
    best.leaf = -1;
    best.orig = 0x7fffffff;
    best.front = false;
    sp = 0;
    steps = 0;
    node = sc.T > 0 ? 0 : FIPT_DONE;
}

// STATS: an instrumented build of the same code that adds its rays, node
// visits and triangle tests to stats[0..2] and raises stats[3] to its
// deepest stack.
template <bool PER_SAMPLE, bool STATS>
__global__ void __launch_bounds__(REFINE_THREADS, REFINE_MINB)
k_refine(SceneView sc, const fipt_query* __restrict__ q, int64_t N, RefineArgs R, float* __restrict__ Ld,
         float* __restrict__ Ls0, float* __restrict__ Ls1, float* __restrict__ per_sample,
         int32_t* status, unsigned long long* stats) {
    constexpr unsigned FULL = 0xffffffffu;
    __shared__ int stk[STACK_DEPTH * REFINE_THREADS];
    int* stack = stk + threadIdx.x;
    const BakeArgs& A = R.A;
    const int K = A.K, L = 1 + K;
    const int64_t g = blockIdx.x * (int64_t)REFINE_THREADS + threadIdx.x;
    const int64_t w = g >> 5;
    const int lobe = (int)(w % L);
    const int64_t p = (w / L) * 32 + (int)(g & 31);
    if ((w / L) * 32 >= N) return;          // whole warp past the end
    const bool valid = p < N;
    const float eps = sc.cst->eps;
    const int n_emit = sc.cst->n_emit;
    const double A_emit = sc.cst->A_emit;
    const bool mis = R.mis && n_emit > 0;
    // the emitter choice compares FP64 cumulative areas (exact selection);
    // the area-measure pdfs dist^2 / (A cos) feed weights only, in FP32
    const float A_emit_f = (float)A_emit;
    const uint32_t pid = A.point_base + (uint32_t)p;
    float a2 = 0.0f;
    if (lobe > 0) {
        float sg = A.sigma[0];
#pragma unroll
        for (int k = 1; k < FIPT_MAX_K; ++k)
            if (lobe - 1 == k) sg = A.sigma[k];
        const float al = sg * sg;
        a2 = al * al;
    }
    int S = 0;
    if (valid) {
        const float2* qp = reinterpret_cast<const float2*>(q + p);
        const float2 q1 = qp[1], q2 = qp[2], q3 = qp[3], q4 = qp[4];
        const float nl = 1.0f / sqrtf(q1.y * q1.y + q2.x * q2.x + q2.y * q2.y);
        const float wl = 1.0f / sqrtf(q3.x * q3.x + q3.y * q3.y + q4.x * q4.x);
        const float mu = (q1.y * nl) * (q3.x * wl) + (q2.x * nl) * (q3.y * wl) + (q2.y * nl) * (q4.x * wl);
        // specular terms of points seen at grazing angles are defined as zero
        S = (lobe > 0 && mu <= 1e-2f) ? 0 : (lobe == 0 ? A.spp_d : A.spp_s);
    }

    // per-lane path state
    int kind = K_NONE, s = 0, depth = 0, skip = -1, tgt = -1, vleaf = -1;
    float dx = 0.0f, dy = 0.0f, dz = 1.0f;            // current path direction
    float b0 = 1.0f, b1 = 1.0f, b2 = 1.0f;            // path throughput
    float l0 = 0.0f, l1 = 0.0f, l2 = 0.0f;            // path radiance
    float W0 = 1.0f, W1 = 0.0f, pdf_prev = 0.0f;
    float sw0 = 0.0f, sw1 = 0.0f, sw2 = 0.0f;         // shadow-ray weights
    float a0 = 0.0f, a1 = 0.0f, a2s = 0.0f, a3 = 0.0f, a4 = 0.0f, a5 = 0.0f;   // sums over samples
    float c0 = 0.0f, c1 = 0.0f, c2 = 0.0f, c3 = 0.0f, c4 = 0.0f, c5 = 0.0f;    // this sample (per-sample output)
    TraceRay r;
    BestHit best;
    best.t = FINF;
    best.leaf = -1;
    best.orig = 0x7fffffff;
    best.front = false;
    r = make_ray(0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f);
    int node = FIPT_DONE, pleaf = -1, sp = 0, steps = 0;
    WalkStats ws;
    unsigned long long n_rays = 0;

#define FIPT_ADD6(cv, av, v)       \
    do {                           \
        if (PER_SAMPLE) cv += (v); \
        else av += (v);            \
    } while (0)

    for (;;) {
        const bool idle = node == FIPT_DONE && pleaf < 0;
        const bool need = idle && (kind != K_NONE || s < S);
        const unsigned m_need = __ballot_sync(FULL, need);
        const unsigned m_busy = __ballot_sync(FULL, !idle);
        if ((m_need | m_busy) == 0) break;
        if (m_need != 0 && (m_busy == 0 || __popc(m_need) >= FIPT_REFINE_REFILL) && need) {
            // ---------------- consume the finished ray
            int act = A_START;
            float xox = 0.0f, xoy = 0.0f, xoz = 0.0f;     // origin of a vertex's continuation
            if (kind == K_S0) {
                if (best.leaf == tgt) {
                    const float4 le = __ldg(sc.shade + 2 * tgt);
                    FIPT_ADD6(c0, a0, sw0 * le.x); FIPT_ADD6(c1, a1, sw0 * le.y); FIPT_ADD6(c2, a2s, sw0 * le.z);
                    FIPT_ADD6(c3, a3, sw1 * le.x); FIPT_ADD6(c4, a4, sw1 * le.y); FIPT_ADD6(c5, a5, sw1 * le.z);
                }
                act = A_MAIN;
            } else if (kind == K_SV) {
                if (best.leaf == tgt) {
                    const float4 le = __ldg(sc.shade + 2 * tgt);
                    l0 += sw0 * le.x; l1 += sw1 * le.y; l2 += sw2 * le.z;
                }
                xox = r.ox; xoy = r.oy; xoz = r.oz;
                act = A_VERTEX_BSDF;
            } else if (kind == K_PATH) {
                act = A_END_PATH;
                if (best.leaf < 0) {
                    if (sc.env) {
                        const float3 e = env_lookup(sc, dx, dy, dz);
                        l0 += b0 * e.x; l1 += b1 * e.y; l2 += b2 * e.z;
                    }
                } else {
                    const int leaf = best.leaf;
                    const float hx = r.ox + best.t * dx, hy = r.oy + best.t * dy, hz = r.oz + best.t * dz;
                    const float4 le = __ldg(sc.shade + 2 * leaf);
                    if (is_emitter(le)) {
                        if (best.front) {
                            float wgt = 1.0f;
                            if (mis) {
                                const float3 ne = leaf_normal(sc, leaf);
                                const float ce = fabsf(dx * ne.x + dy * ne.y + dz * ne.z);
                                const float pl = best.t * best.t / (A_emit_f * ce);
                                wgt = pdf_prev * pdf_prev / (pdf_prev * pdf_prev + pl * pl);
                            }
                            l0 += b0 * wgt * le.x; l1 += b1 * wgt * le.y; l2 += b2 * wgt * le.z;
                        }
                    } else if (__ldg(&sc.mats[2 * leaf].w) > R.sigma_c) {
                        float3 ca;
                        if (sc.vox) {
                            ca = voxel_lookup(sc, hx, hy, hz);
                        } else {
                            const float4 c4 = __ldg(sc.shade + 2 * leaf + 1);
                            ca = make_float3(c4.x, c4.y, c4.z);
                        }
                        l0 += b0 * ca.x; l1 += b1 * ca.y; l2 += b2 * ca.z;
                    } else if (depth <= R.max_depth) {
                        // a smooth surface: a path vertex
                        float3 nv = leaf_normal(sc, leaf);
                        if (nv.x * dx + nv.y * dy + nv.z * dz > 0.0f) nv = make_float3(-nv.x, -nv.y, -nv.z);
                        xox = hx + eps * nv.x; xoy = hy + eps * nv.y; xoz = hz + eps * nv.z;
                        vleaf = leaf;
                        skip = best.orig;
                        act = A_VERTEX_BSDF;
                        if (mis) {
                            const float3 wv = make_float3(-dx, -dy, -dz);
                            const float mu_v = nv.x * wv.x + nv.y * wv.y + nv.z * wv.z;
                            const Mat M = vertex_mat(sc, leaf, mu_v);
                            float3 y;
                            const uint32_t lc = (uint32_t)lobe | ((uint32_t)depth << 9) | 0x100u;
                            const int e = emitter_sample(sc, n_emit, A_emit, u4(pid, (uint32_t)s, lc, A), y);
                            float ex = y.x - xox, ey = y.y - xoy, ez = y.z - xoz;
                            const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                            ex /= dist; ey /= dist; ez /= dist;
                            const float3 ne = leaf_normal(sc, e);
                            const float ce = -(ex * ne.x + ey * ne.y + ez * ne.z);
                            if (ce > 0.0f) {
                                float f[3], pb;
                                vertex_brdf(M, nv, wv, make_float3(ex, ey, ez), mu_v, f, pb);
                                if (f[0] > 0.0f || f[1] > 0.0f || f[2] > 0.0f) {
                                    const float pl = dist * dist / (A_emit_f * ce);
                                    const float wgt = pl * pl / (pl * pl + pb * pb);
                                    sw0 = b0 * wgt * f[0] / pl;
                                    sw1 = b1 * wgt * f[1] / pl;
                                    sw2 = b2 * wgt * f[2] / pl;
                                    tgt = e;
                                    start_ray(r, best, node, sp, steps, sc, xox, xoy, xoz, ex, ey, ez,
                                              1.001f * dist + eps);
                                    if (STATS) ++n_rays;
                                    kind = K_SV;
                                    act = A_RAY;
                                }
                            }
                        }
                    }
                }
            }
            // ---------------- set up the next ray
            while (act != A_RAY) {
                if (act == A_VERTEX_BSDF) {            // BRDF sample at path vertex `depth`
                    float3 nv = leaf_normal(sc, vleaf);
                    if (nv.x * dx + nv.y * dy + nv.z * dz > 0.0f) nv = make_float3(-nv.x, -nv.y, -nv.z);
                    const float3 wv = make_float3(-dx, -dy, -dz);
                    const float mu_v = nv.x * wv.x + nv.y * wv.y + nv.z * wv.z;
                    const Mat M = vertex_mat(sc, vleaf, mu_v);
                    const float4 u = u4(pid, (uint32_t)s, (uint32_t)lobe | ((uint32_t)depth << 9), A);
                    float3 tb, bb;
                    onb(nv.x, nv.y, nv.z, tb, bb);
                    float3 wi, hh = make_float3(0.0f, 0.0f, 1.0f);
                    float sin2h = 0.0f, sn, cs;
                    sincospif(2.0f * u.y, &sn, &cs);
                    const bool glossy = !(u.z < M.Pd);
                    if (!glossy) {
                        const float rr = sqrtf(u.x);
                        wi = to_world(tb, bb, nv, rr * cs, rr * sn, sqrtf(1.0f - u.x));
                    } else {
                        const float om = 1.0f - u.x;
                        const float den = om + M.a2 * u.x;
                        sin2h = M.a2 * u.x / den;
                        const float ch = sqrtf(om / den), sh = sqrtf(sin2h);
                        hh = to_world(tb, bb, nv, sh * cs, sh * sn, ch);
                        const float c = wv.x * hh.x + wv.y * hh.y + wv.z * hh.z;
                        wi = make_float3(2.0f * c * hh.x - wv.x, 2.0f * c * hh.y - wv.y, 2.0f * c * hh.z - wv.z);
                    }
                    float f[3], pdf;
                    vertex_brdf(M, nv, wv, wi, mu_v, f, pdf, glossy, hh, sin2h);
                    if (pdf <= 0.0f) {
                        act = A_END_PATH;
                    } else {
                        b0 *= f[0] / pdf; b1 *= f[1] / pdf; b2 *= f[2] / pdf;
                        start_ray(r, best, node, sp, steps, sc, xox, xoy, xoz, wi.x, wi.y, wi.z, FINF);
                        if (STATS) ++n_rays;
                        dx = wi.x; dy = wi.y; dz = wi.z;
                        pdf_prev = pdf;
                        ++depth;
                        kind = K_PATH;
                        act = A_RAY;
                        break;
                    }
                }
                if (act == A_END_PATH) {
                    FIPT_ADD6(c0, a0, W0 * l0); FIPT_ADD6(c1, a1, W0 * l1); FIPT_ADD6(c2, a2s, W0 * l2);
                    FIPT_ADD6(c3, a3, W1 * l0); FIPT_ADD6(c4, a4, W1 * l1); FIPT_ADD6(c5, a5, W1 * l2);
                    act = A_END_SAMPLE;
                }
                if (act == A_END_SAMPLE) {
                    if (PER_SAMPLE) {
                        float* ps = per_sample + ((size_t)(p * L + lobe) * R.smax + s) * 6;
                        a0 += c0; a1 += c1; a2s += c2; a3 += c3; a4 += c4; a5 += c5;
                        ps[0] = c0; ps[1] = c1; ps[2] = c2; ps[3] = c3; ps[4] = c4; ps[5] = c5;
                    }
                    ++s;
                    act = A_START;
                }
                kind = K_NONE;
                if (act == A_START && s >= S) break;  // this pair is done
                // A_START or A_MAIN: the query point's frame
                const float2* qp = reinterpret_cast<const float2*>(q + p);
                const float2 q0 = qp[0], q1 = qp[1], q2 = qp[2], q3 = qp[3], q4 = qp[4];
                float3 n = make_float3(q1.y, q2.x, q2.y), wo = make_float3(q3.x, q3.y, q4.x);
                {
                    const float il = 1.0f / sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
                    n = make_float3(n.x * il, n.y * il, n.z * il);
                    const float jl = 1.0f / sqrtf(wo.x * wo.x + wo.y * wo.y + wo.z * wo.z);
                    wo = make_float3(wo.x * jl, wo.y * jl, wo.z * jl);
                }
                const float mu_o = n.x * wo.x + n.y * wo.y + n.z * wo.z;
                const float ox = q0.x + eps * n.x, oy = q0.y + eps * n.y, oz = q1.x + eps * n.z;
                const float g1o = lobe > 0 ? smith_g1(mu_o, a2) : 0.0f;
                if (act == A_START) {
                    c0 = c1 = c2 = c3 = c4 = c5 = 0.0f;
                    act = A_MAIN;
                    if (mis) {                         // emitter sample at x
                        float3 y;
                        const int e = emitter_sample(sc, n_emit, A_emit,
                                                     u4(pid, (uint32_t)s, (uint32_t)lobe | 0x100u, A), y);
                        float ex = y.x - ox, ey = y.y - oy, ez = y.z - oz;
                        const float dist = sqrtf(ex * ex + ey * ey + ez * ez);
                        ex /= dist; ey /= dist; ez /= dist;
                        const float3 ne = leaf_normal(sc, e);
                        const float ce = -(ex * ne.x + ey * ne.y + ez * ne.z);
                        const float mu_i = n.x * ex + n.y * ey + n.z * ez;
                        float g0 = 0.0f, g1 = 0.0f, pb = 0.0f;
                        if (ce > 0.0f && mu_i > 0.0f) {
                            if (lobe == 0) {
                                g0 = mu_i / PI_F;
                                pb = g0;
                            } else {
                                float hx = ex + wo.x, hy = ey + wo.y, hz = ez + wo.z;
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
                            const float pl = dist * dist / (A_emit_f * ce);
                            const float wgt = pl * pl / (pl * pl + pb * pb);
                            sw0 = wgt * g0 / pl;
                            sw1 = wgt * g1 / pl;
                            tgt = e;
                            skip = __float_as_int(q4.y);
                            start_ray(r, best, node, sp, steps, sc, ox, oy, oz, ex, ey, ez, 1.001f * dist + eps);
                            if (STATS) ++n_rays;
                            kind = K_S0;
                            act = A_RAY;
                            break;
                        }
                    }
                }
                // A_MAIN: the lobe sample at x (the stage-1 sampler)
                const float4 u = u4(pid, (uint32_t)s, (uint32_t)lobe, A);
                float3 tb, bb;
                onb(n.x, n.y, n.z, tb, bb);
                float sn, cs;
                sincospif(2.0f * u.y, &sn, &cs);
                float3 wi;
                W0 = 1.0f;
                W1 = 0.0f;
                float pb = 0.0f;
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
                    if (mu_i <= 0.0f || c <= 0.0f) {   // a zero sample
                        act = A_END_SAMPLE;
                        continue;
                    }
                    const float wt = smith_g1(mu_i, a2) * g1o * c / (mu_o * ch);
                    const float x1 = 1.0f - c, x2 = x1 * x1, F1 = x2 * x2 * x1;
                    W0 = (1.0f - F1) * wt;
                    W1 = F1 * wt;
                    pb = ggx_d(sin2, cos2, a2) * ch / (4.0f * c);
                }
                b0 = b1 = b2 = 1.0f;
                l0 = l1 = l2 = 0.0f;
                pdf_prev = pb;
                depth = 1;
                skip = __float_as_int(q4.y);
                dx = wi.x; dy = wi.y; dz = wi.z;
                start_ray(r, best, node, sp, steps, sc, ox, oy, oz, wi.x, wi.y, wi.z, FINF);
                if (STATS) ++n_rays;
                kind = K_PATH;
                act = A_RAY;
            }
        }
        // ---------------- inner nodes (speculative), then leaves
        warp_walk<REFINE_THREADS, STATS, true>(sc, r, skip, best, node, pleaf, sp, steps, stack, status, ws);
    }
#undef FIPT_ADD6

    if (STATS) {
        atomicAdd(&stats[0], n_rays);
        atomicAdd(&stats[1], ws.nodes);
        atomicAdd(&stats[2], ws.tris);
        atomicMax(&stats[3], (unsigned long long)ws.max_sp);
    }
    if (!valid) return;
    if (PER_SAMPLE) {
        float* ps = per_sample + (size_t)(p * L + lobe) * R.smax * 6;
        for (int i = S; i < R.smax; ++i)
            for (int c = 0; c < 6; ++c) ps[i * 6 + c] = 0.0f;
    }
    const float fs = (float)(S > 0 ? S : 1);
    if (lobe == 0) {
        Ld[3 * p + 0] = a0 / fs;
        Ld[3 * p + 1] = a1 / fs;
        Ld[3 * p + 2] = a2s / fs;
    } else {
        float* o0 = Ls0 + (p * K + (lobe - 1)) * 3;
        float* o1 = Ls1 + (p * K + (lobe - 1)) * 3;
        o0[0] = a0 / fs; o0[1] = a1 / fs; o0[2] = a2s / fs;
        o1[0] = a3 / fs; o1[1] = a4 / fs; o1[2] = a5 / fs;
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
    FIPT_REQUIRE(!(prm->stats && per_sample), "stats and per_sample cannot be combined");
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
        FIPT_LAUNCH((k_refine<true, false>), blocks(threads, REFINE_THREADS), REFINE_THREADS, 0, st, s->view(),
                    q, N, R, Ld, Ls0, Ls1, per_sample, s->ctx->status, nullptr);
    else if (prm->stats)
        FIPT_LAUNCH((k_refine<false, true>), blocks(threads, REFINE_THREADS), REFINE_THREADS, 0, st, s->view(),
                    q, N, R, Ld, Ls0, Ls1, nullptr, s->ctx->status, prm->stats);
    else
        FIPT_LAUNCH((k_refine<false, false>), blocks(threads, REFINE_THREADS), REFINE_THREADS, 0, st,
                    s->view(), q, N, R, Ld, Ls0, Ls1, nullptr, s->ctx->status, nullptr);
    FIPT_LAUNCHED("bake_refine");
    return FIPT_OK;
}
