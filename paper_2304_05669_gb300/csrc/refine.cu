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
//
// Organisation (wavefront path tracing, Laine, Karras and Aila 2013).  One
// slot per sample (point, lobe, s); a chunk of at most FIPT_RF_SLOT_CAP
// slots keeps its path state in the caller's workspace, 16-byte records
// per slot.  Per chunk:
//   k_rf_gen     sets up every slot at its query point: the emitter sample
//                at x (a shadow ray) and the lobe sample (the first path
//                segment), and queues both rays;
//   k_rf_trace   closest hit of every queued ray: a persistent kernel whose
//                warps draw rays from the queue and walk the tree with the
//                stage-1 bake's speculative, warp-refilled traversal (stack
//                in local memory, as the bake's);
//   k_rf_shade   consumes a slot's hits (the shadow ray first, then the
//                path segment), and at a smooth surface queues the vertex's
//                shadow ray and its next segment together (the BRDF sample
//                does not depend on the shadow ray's outcome);
//   k_rf_reduce  sums each (point, lobe)'s samples in sample order.
// trace + shade run once per path depth (max_depth + 1 times).  Every
// slot's arithmetic is the same sequence whatever the queue order, so the
// results do not depend on scheduling.  The traversal kernel carries only
// a ray; the shading state stays in HBM, and each kernel runs its lanes
// through one kind of work.
#include "fipt_internal.cuh"

namespace {

#ifndef FIPT_RF_TRACE_THREADS
#define FIPT_RF_TRACE_THREADS 64
#endif
#ifndef FIPT_RF_TRACE_MINB
#define FIPT_RF_TRACE_MINB 24        // resident traversal blocks per SM (40 registers)
#endif
#ifndef FIPT_RF_REFILL
#define FIPT_RF_REFILL 24            // idle lanes that make a warp draw new rays
#endif
#ifndef FIPT_RF_SLOT_CAP
#define FIPT_RF_SLOT_CAP (1 << 24)   // samples per chunk (184 B of workspace each)
#endif
#ifndef FIPT_RF_SHADE_MINB
#define FIPT_RF_SHADE_MINB 3         // resident shading blocks per SM the register budget must allow
#endif
constexpr int RF_TRACE_THREADS = FIPT_RF_TRACE_THREADS;
constexpr int RF_SHADE_THREADS = 256;
constexpr int64_t RF_SLOT_CAP = FIPT_RF_SLOT_CAP;
constexpr float PI_F = 3.14159265358979f;

struct RefineArgs {
    BakeArgs A;
    float sigma_c;
    int max_depth;
    int mis;
    int smax;               // stride of the per-sample output
    int per_pt;             // samples per point: spp_d + K * spp_s
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

// Unit face normal (not oriented) of the triangle with vertices p0, p1, p2.
__device__ __forceinline__ float3 tri_normal(float4 p0, float4 p1, float4 p2) {
    const float e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
    const float e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
    float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
    const float il = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
    return make_float3(nx * il, ny * il, nz * il);
}

// Unit face normal of a leaf (not oriented).
__device__ __forceinline__ float3 leaf_normal(const SceneView& sc, int leaf) {
    return tri_normal(__ldg(sc.tris + 3 * leaf), __ldg(sc.tris + 3 * leaf + 1), __ldg(sc.tris + 3 * leaf + 2));
}

struct Mat {
    float kd[3], ks[3];
    float a2;
    float Pd;
    bool spec;
};

// Eq. 1's k_d, k_s, alpha^2 and the diffuse-lobe probability from a leaf's
// material records m0 = (albedo, roughness), m1 = (metallic, ...).
__device__ __forceinline__ Mat vertex_mat(float4 m0, float4 m1, float mu_o) {
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

// ---------------------------------------------------------------- path state
// Flags word of a slot: bits 0-15 the path depth (segments issued), then
// whether a path segment or a shadow ray is queued, whether that shadow ray
// starts at the query point (its weights then go to the sample's value, not
// to the path radiance), and whether the path is live (its radiance not
// yet added to the sample's value).
constexpr uint32_t F_DEPTH = 0xffffu;
constexpr uint32_t F_PATH = 1u << 16, F_SHADOW = 1u << 17, F_AT_X = 1u << 18, F_LIVE = 1u << 19;

struct RfState {
    float4* org;        // [P] origin of the slot's rays (xyz), the triangle they skip (int bits)
    float4* dir;        // [2P] ray 2j: path segment, 2j+1: shadow ray; direction (xyz), t_max
    int4* hit;          // [2P] t (float bits), leaf (-1: none), original triangle id, front face
    float4* bp;         // [P] path throughput (rgb), pdf of the last BRDF sample
    float4* lw;         // [P] path radiance (rgb), W0
    float4* c0;         // [P] sample value for L_d / L_s0 (rgb), W1
    float4* c1;         // [P] sample value for L_s1 (rgb), flags (int bits)
    float4* sw;         // [P] shadow-ray weights (rgb), target emitter leaf (int bits)
    uint32_t* act[2];   // slots with queued rays, by wave parity
    uint32_t* tq[2];    // queued ray ids, by wave parity
    uint32_t* cnt;      // wave w: [4w] rays queued, [4w+1] rays taken, [4w+2] slots active
};

struct RfChunk {
    const fipt_query* q;    // the chunk's first query
    int64_t p0;             // index of that query in the call
    int64_t n_pts;          // points in the chunk
    int64_t P;              // slots: n_pts * per_pt
};

// (point within the chunk, lobe, sample) of slot j.  A point's samples in
// order are its spp_d diffuse samples, then spp_s of each roughness level;
// slot j holds sample r = j / n_pts of point j mod n_pts, so the 32 slots
// of a warp are 32 points at one lobe and sample index: their first rays
// leave through the same stratum of directions (reading 26) and walk the
// tree alike.
__device__ __forceinline__ void slot_decode(int64_t j, const RefineArgs& R, int64_t n_pts, int64_t& pc,
                                            int& lobe, int& s) {
    const int64_t rr = j / n_pts;
    pc = j - rr * n_pts;
    int r = (int)rr;
    if (r < R.A.spp_d) {
        lobe = 0;
        s = r;
    } else {
        r -= R.A.spp_d;
        lobe = 1 + r / R.A.spp_s;
        s = r - (lobe - 1) * R.A.spp_s;
    }
}

// Appends v to list for every lane with pred (one atomic per warp); all 32
// lanes of the warp call it together.
__device__ __forceinline__ void warp_append(uint32_t* list, uint32_t* count, bool pred, uint32_t v) {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// ---------------------------------------------------------------- generation
// Every slot at its query point: the emitter sample at x (MIS) and the
// lobe sample of the stage-1 bake, queued as rays of wave 0.
__global__ void __launch_bounds__(RF_SHADE_THREADS)
k_rf_gen(SceneView sc, RfChunk C, RefineArgs R, RfState st) {
    const BakeArgs& A = R.A;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * RF_SHADE_THREADS;
    const float eps = sc.cst->eps;
    const int n_emit = sc.cst->n_emit;
    const double A_emit = sc.cst->A_emit;
    const bool mis = R.mis && n_emit > 0;
    // the emitter choice compares FP64 cumulative areas (exact selection);
    // the area-measure pdfs dist^2 / (A cos) feed weights only, in FP32
    const float A_emit_f = (float)A_emit;
    for (int64_t base = (int64_t)blockIdx.x * RF_SHADE_THREADS + (threadIdx.x & ~31); base < C.P;
         base += stride) {
        const int64_t j = base + lane;
        bool qpath = false, qshadow = false;
        if (j < C.P) {
            int64_t pc;
            int lobe, s;
            slot_decode(j, R, C.n_pts, pc, lobe, s);
            const float2* qp = reinterpret_cast<const float2*>(C.q + pc);
            const float2 q0 = qp[0], q1 = qp[1], q2 = qp[2], q3 = qp[3], q4 = qp[4];
            float3 n = make_float3(q1.y, q2.x, q2.y), wo = make_float3(q3.x, q3.y, q4.x);
            {
                const float il = 1.0f / sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
                n = make_float3(n.x * il, n.y * il, n.z * il);
                const float jl = 1.0f / sqrtf(wo.x * wo.x + wo.y * wo.y + wo.z * wo.z);
                wo = make_float3(wo.x * jl, wo.y * jl, wo.z * jl);
            }
            const float mu_o = n.x * wo.x + n.y * wo.y + n.z * wo.z;
            // specular terms of points seen at grazing angles are defined as zero
            const bool grazing = lobe > 0 && mu_o <= 1e-2f;
            float4 C0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), C1 = C0;
            uint32_t flags = 0;
            if (!grazing) {
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
                const uint32_t pid = A.point_base + (uint32_t)(C.p0 + pc);
                const float ox = q0.x + eps * n.x, oy = q0.y + eps * n.y, oz = q1.x + eps * n.z;
                st.org[j] = make_float4(ox, oy, oz, q4.y);         // q4.y: the query's triangle
                if (mis) {                                          // emitter sample at x
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
                        st.sw[j] = make_float4(wgt * g0 / pl, wgt * g1 / pl, 0.0f, __int_as_float(e));
                        st.dir[2 * j + 1] = make_float4(ex, ey, ez, 1.001f * dist + eps);
                        flags |= F_SHADOW | F_AT_X;
                        qshadow = true;
                    }
                }
                // the lobe sample at x (the stage-1 sampler, stratified as there)
                float4 u = u4(pid, (uint32_t)s, (uint32_t)lobe, A);
                strat_uv((uint32_t)s, lobe == 0 ? A.spp_d : A.spp_s, lobe == 0 ? A.nx_d : A.nx_s, u.x, u.y);
                float3 tb, bb;
                onb(n.x, n.y, n.z, tb, bb);
                float sn, cs;
                sincospif(2.0f * u.y, &sn, &cs);
                float3 wi;
                float W0 = 1.0f, W1 = 0.0f, pb = 0.0f;
                bool ok = true;
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
                    if (mu_i <= 0.0f || c <= 0.0f) {    // a zero sample: no path
                        ok = false;
                    } else {
                        const float wt = smith_g1(mu_i, a2) * g1o * c / (mu_o * ch);
                        const float x1 = 1.0f - c, x2 = x1 * x1, F1 = x2 * x2 * x1;
                        W0 = (1.0f - F1) * wt;
                        W1 = F1 * wt;
                        pb = ggx_d(sin2, cos2, a2) * ch / (4.0f * c);
                    }
                }
                if (ok) {
                    st.dir[2 * j] = make_float4(wi.x, wi.y, wi.z, FINF);
                    st.bp[j] = make_float4(1.0f, 1.0f, 1.0f, pb);
                    st.lw[j] = make_float4(0.0f, 0.0f, 0.0f, W0);
                    C0.w = W1;
                    flags |= F_PATH | F_LIVE | 1u;
                    qpath = true;
                }
            }
            C1.w = __uint_as_float(flags);
            st.c0[j] = C0;
            st.c1[j] = C1;
        }
        warp_append(st.act[0], st.cnt + 2, qpath || qshadow, (uint32_t)j);
        warp_append(st.tq[0], st.cnt + 0, qpath, (uint32_t)(2 * j));
        warp_append(st.tq[0], st.cnt + 0, qshadow, (uint32_t)(2 * j + 1));
    }
}

// ---------------------------------------------------------------- traversal
// Closest hit of every ray queued for wave w.  Persistent: each warp draws
// rays from the queue (one atomic per refill) whenever FIPT_RF_REFILL of
// its lanes are idle, or all of them, and walks the tree with the stage-1
// bake's speculative loop.
//
// A shadow ray only asks whether its target emitter triangle is the
// closest hit within t_max (just past the sampled point), ties going to the
// lower triangle id.  The target is tested first, with the same watertight
// test: if its (t, id) is not below (t_max, INT_MAX), or it is the skipped
// triangle, no walk can make it the closest hit and the ray ends there.
// Otherwise it seeds the closest hit and the walk stops at the first
// triangle that improves on it (a blocker: the answer is no).  Culling
// against the seeded t keeps every box that can hold a blocker, so the
// answer is the one a full closest-hit walk gives; only the recorded leaf
// of a blocked ray may differ (any blocker instead of the nearest).
//
// STATS: an instrumented build that adds its rays, node visits and
// triangle tests to stats[0..2] and raises stats[3] to its deepest stack.
template <bool STATS>
__global__ void __launch_bounds__(RF_TRACE_THREADS, FIPT_RF_TRACE_MINB)
k_rf_trace(SceneView sc, RfState st, int w, int32_t* status, unsigned long long* stats) {
    constexpr unsigned FULL = 0xffffffffu;
    int stack[STACK_DEPTH];             // local memory, as the stage-1 bake's
    const uint32_t* __restrict__ queue = st.tq[w & 1];
    uint32_t* cnt = st.cnt + 4 * w;
    const uint32_t n = cnt[0];
    if (n == 0) return;
    const int lane = threadIdx.x & 31;
    int rid = -1, skip = -1;
    bool drained = false, shadow = false;
    TraceRay r = make_ray(0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f);
    BestHit best;
    best.t = FINF;
    best.leaf = -1;
    best.orig = 0x7fffffff;
    best.front = false;
    int node = FIPT_DONE, pleaf = -1, sp = 0, steps = 0;
    WalkStats ws;
    unsigned long long n_rays = 0;
    for (;;) {
        const bool idle = node == FIPT_DONE && pleaf < 0;
        if (idle && rid >= 0) {
            st.hit[rid] = make_int4(__float_as_int(best.t), best.leaf, best.orig, best.front ? 1 : 0);
            rid = -1;
        }
        const bool need = idle && !drained;
        const unsigned m_need = __ballot_sync(FULL, need);
        const unsigned m_busy = __ballot_sync(FULL, !idle);
        if ((m_need | m_busy) == 0) break;
        if (m_need != 0 && (m_busy == 0 || __popc(m_need) >= FIPT_RF_REFILL)) {
            const int leader = __ffs(m_need) - 1;
            uint32_t b = 0;
            if (lane == leader) b = atomicAdd(cnt + 1, (uint32_t)__popc(m_need));
            b = __shfl_sync(FULL, b, leader);
            if (need) {
                const uint32_t i = b + __popc(m_need & ((1u << lane) - 1u));
                if (i < n) {
                    rid = (int)__ldg(queue + i);
                    const float4 o = __ldg(st.org + (rid >> 1)), d = __ldg(st.dir + rid);
                    r = make_ray(o.x, o.y, o.z, d.x, d.y, d.z);
                    skip = __float_as_int(o.w);
                    best.t = d.w;
                    best.leaf = -1;
                    best.orig = 0x7fffffff;
                    best.front = false;
                    sp = 0;
                    steps = 0;
                    node = sc.T > 0 ? 0 : FIPT_DONE;
                    if (STATS) ++n_rays;
                    shadow = (rid & 1) != 0;
                    if (shadow) {                  // settle the target first
                        const int tgt = __float_as_int(__ldg(&st.sw[rid >> 1].w));
                        const float4 p0 = __ldg(sc.tris + 3 * tgt);
                        const int orig = __float_as_int(p0.w);
                        float t;
                        bool fr;
                        if (STATS) ++ws.tris;
                        if (orig != skip &&
                            tri_intersect(r, p0, __ldg(sc.tris + 3 * tgt + 1), __ldg(sc.tris + 3 * tgt + 2), t, fr) &&
                            (t < best.t || (t == best.t && orig < best.orig))) {
                            best.t = t;
                            best.leaf = tgt;
                            best.orig = orig;
                            best.front = fr;
                        } else {
                            node = FIPT_DONE;      // unlit whatever else the ray meets
                        }
                    }
                } else {
                    drained = true;      // the queue is empty for good
                }
            }
        }
        warp_walk<1, STATS, true>(sc, r, skip, best, node, pleaf, sp, steps, stack, status, ws,
                                                 shadow);
    }
    if (STATS) {
        atomicAdd(&stats[0], n_rays);
        atomicAdd(&stats[1], ws.nodes);
        atomicAdd(&stats[2], ws.tris);
        atomicMax(&stats[3], (unsigned long long)ws.max_sp);
    }
}

// ---------------------------------------------------------------- shading
// Every slot active in wave w: the shadow ray's emitter (if it was hit
// first), then the path segment's hit: a miss (environment), an emitter
// (L_e of the front face, MIS-weighted), a rough surface (L'), or a smooth
// one, where the vertex's emitter sample and BRDF sample are queued for
// wave w + 1.  A slot with nothing queued adds its path radiance
// (W0, W1 times l) to its value and leaves the lists.
__global__ void __launch_bounds__(RF_SHADE_THREADS, FIPT_RF_SHADE_MINB)
k_rf_shade(SceneView sc, RfChunk C, RefineArgs R, RfState st, int w) {
    const BakeArgs& A = R.A;
    const int lane = threadIdx.x & 31;
    const uint32_t* __restrict__ act = st.act[w & 1];
    uint32_t* nact = st.act[(w + 1) & 1];
    uint32_t* ntq = st.tq[(w + 1) & 1];
    uint32_t* ncnt = st.cnt + 4 * (w + 1);
    const int64_t n = st.cnt[4 * w + 2];
    const int64_t stride = (int64_t)gridDim.x * RF_SHADE_THREADS;
    const float eps = sc.cst->eps;
    const int n_emit = sc.cst->n_emit;
    const double A_emit = sc.cst->A_emit;
    const bool mis = R.mis && n_emit > 0;
    const float A_emit_f = (float)A_emit;
    for (int64_t base = (int64_t)blockIdx.x * RF_SHADE_THREADS + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t i = base + lane;
        bool qpath = false, qshadow = false;
        uint32_t j = 0;
        if (i < n) {
            j = act[i];
            int64_t pc;
            int lobe, s;
            slot_decode(j, R, C.n_pts, pc, lobe, s);
            const uint32_t pid = A.point_base + (uint32_t)(C.p0 + pc);
            float4 C0 = st.c0[j], C1 = st.c1[j], LW = st.lw[j];
            // the slot's other records, loaded together whether or not a ray
            // of their kind was queued (they are unused then)
            const float4 SW = st.sw[j], D = st.dir[2 * j], O = st.org[j];
            const int4 hs = st.hit[2 * j + 1], h = st.hit[2 * j];
            const float4 BP = st.bp[j];
            const uint32_t f_in = __float_as_uint(C1.w);
            uint32_t depth = f_in & F_DEPTH;
            uint32_t flags = f_in & F_LIVE;
            if (f_in & F_SHADOW) {                      // the shadow ray queued last wave
                const int tgt = __float_as_int(SW.w);
                if (hs.y == tgt) {
                    const float4 le = __ldg(sc.shade + 2 * tgt);
                    if (f_in & F_AT_X) {
                        C0.x += SW.x * le.x; C0.y += SW.x * le.y; C0.z += SW.x * le.z;
                        C1.x += SW.y * le.x; C1.y += SW.y * le.y; C1.z += SW.y * le.z;
                    } else {
                        LW.x += SW.x * le.x; LW.y += SW.y * le.y; LW.z += SW.z * le.z;
                    }
                }
            }
            if (f_in & F_PATH) {                        // the path segment queued last wave
                const float dx = D.x, dy = D.y, dz = D.z;
                if (h.y < 0) {
                    if (sc.env) {
                        const float3 e = env_lookup(sc, dx, dy, dz);
                        LW.x += BP.x * e.x; LW.y += BP.y * e.y; LW.z += BP.z * e.z;
                    }
                } else {
                    const int leaf = h.y;
                    const float t = __int_as_float(h.x);
                    const float hx = O.x + t * dx, hy = O.y + t * dy, hz = O.z + t * dz;
                    // everything the hit's shading can need, loaded together
                    const float4 le = __ldg(sc.shade + 2 * leaf), c4 = __ldg(sc.shade + 2 * leaf + 1);
                    const float4 m0 = __ldg(sc.mats + 2 * leaf), m1 = __ldg(sc.mats + 2 * leaf + 1);
                    const float4 p0 = __ldg(sc.tris + 3 * leaf), p1 = __ldg(sc.tris + 3 * leaf + 1),
                                 p2 = __ldg(sc.tris + 3 * leaf + 2);
                    if (is_emitter(le)) {
                        if (h.w) {
                            float wgt = 1.0f;
                            if (mis) {
                                const float3 ne = tri_normal(p0, p1, p2);
                                const float ce = fabsf(dx * ne.x + dy * ne.y + dz * ne.z);
                                const float pl = t * t / (A_emit_f * ce);
                                wgt = BP.w * BP.w / (BP.w * BP.w + pl * pl);
                            }
                            LW.x += BP.x * wgt * le.x; LW.y += BP.y * wgt * le.y; LW.z += BP.z * wgt * le.z;
                        }
                    } else if (m0.w > R.sigma_c) {
                        const float3 ca = sc.vox ? voxel_lookup(sc, hx, hy, hz) : make_float3(c4.x, c4.y, c4.z);
                        LW.x += BP.x * ca.x; LW.y += BP.y * ca.y; LW.z += BP.z * ca.z;
                    } else if ((int)depth <= R.max_depth) {
                        // a smooth surface: path vertex `depth`
                        float3 nv = tri_normal(p0, p1, p2);
                        if (nv.x * dx + nv.y * dy + nv.z * dz > 0.0f) nv = make_float3(-nv.x, -nv.y, -nv.z);
                        const float xox = hx + eps * nv.x, xoy = hy + eps * nv.y, xoz = hz + eps * nv.z;
                        st.org[j] = make_float4(xox, xoy, xoz, __int_as_float(h.z));
                        const float3 wv = make_float3(-dx, -dy, -dz);
                        const float mu_v = nv.x * wv.x + nv.y * wv.y + nv.z * wv.z;
                        const Mat M = vertex_mat(m0, m1, mu_v);
                        const uint32_t lc = (uint32_t)lobe | (depth << 9);
                        if (mis) {                      // emitter sample at the vertex
                            float3 y;
                            const int e = emitter_sample(sc, n_emit, A_emit, u4(pid, (uint32_t)s, lc | 0x100u, A), y);
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
                                    st.sw[j] = make_float4(BP.x * wgt * f[0] / pl, BP.y * wgt * f[1] / pl,
                                                           BP.z * wgt * f[2] / pl, __int_as_float(e));
                                    st.dir[2 * j + 1] = make_float4(ex, ey, ez, 1.001f * dist + eps);
                                    flags |= F_SHADOW;
                                    qshadow = true;
                                }
                            }
                        }
                        // BRDF sample at the vertex
                        const float4 u = u4(pid, (uint32_t)s, lc, A);
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
                        if (pdf > 0.0f) {
                            st.bp[j] = make_float4(BP.x * (f[0] / pdf), BP.y * (f[1] / pdf), BP.z * (f[2] / pdf), pdf);
                            st.dir[2 * j] = make_float4(wi.x, wi.y, wi.z, FINF);
                            ++depth;
                            flags |= F_PATH;
                            qpath = true;
                        }
                    }
                }
            }
            if (!qpath && !qshadow && (flags & F_LIVE)) {   // the path is over
                const float W0 = LW.w, W1 = C0.w;
                C0.x += W0 * LW.x; C0.y += W0 * LW.y; C0.z += W0 * LW.z;
                C1.x += W1 * LW.x; C1.y += W1 * LW.y; C1.z += W1 * LW.z;
                flags &= ~F_LIVE;
            }
            C1.w = __uint_as_float(flags | depth);
            st.c0[j] = C0;
            st.c1[j] = C1;
            st.lw[j] = LW;
        }
        warp_append(nact, ncnt + 2, qpath || qshadow, j);
        warp_append(ntq, ncnt + 0, qpath, 2 * j);
        warp_append(ntq, ncnt + 0, qshadow, 2 * j + 1);
    }
}

// ---------------------------------------------------------------- reduction
// Each (point, lobe) of the chunk: the mean of its samples' values, summed
// in sample order; PER_SAMPLE also writes every sample's value (zeros past
// the lobe's sample count).
template <bool PER_SAMPLE>
__global__ void __launch_bounds__(RF_SHADE_THREADS)
k_rf_reduce(RfChunk C, RefineArgs R, RfState st, float* __restrict__ Ld, float* __restrict__ Ls0,
            float* __restrict__ Ls1, float* __restrict__ per_sample) {
    const int K = R.A.K, L = 1 + K;
    const int64_t t = blockIdx.x * (int64_t)RF_SHADE_THREADS + threadIdx.x;
    if (t >= C.n_pts * L) return;
    const int lobe = (int)(t / C.n_pts);          // neighbouring threads: neighbouring points
    const int64_t pc = t - lobe * C.n_pts;
    const int64_t p = C.p0 + pc;
    const int S = lobe == 0 ? R.A.spp_d : R.A.spp_s;
    const int64_t r0 = lobe == 0 ? 0 : R.A.spp_d + (int64_t)(lobe - 1) * R.A.spp_s;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f, a4 = 0.0f, a5 = 0.0f;
    float* ps = PER_SAMPLE ? per_sample + (size_t)(p * L + lobe) * R.smax * 6 : nullptr;
    for (int s = 0; s < S; ++s) {
        const int64_t j = (r0 + s) * C.n_pts + pc;
        const float4 x = st.c0[j], y = st.c1[j];
        a0 += x.x; a1 += x.y; a2 += x.z;
        a3 += y.x; a4 += y.y; a5 += y.z;
        if (PER_SAMPLE) {
            float* o = ps + (size_t)s * 6;
            o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = y.x; o[4] = y.y; o[5] = y.z;
        }
    }
    if (PER_SAMPLE)
        for (int s = S; s < R.smax; ++s)
            for (int c = 0; c < 6; ++c) ps[(size_t)s * 6 + c] = 0.0f;
    const float fs = (float)S;
    if (lobe == 0) {
        Ld[3 * p + 0] = a0 / fs;
        Ld[3 * p + 1] = a1 / fs;
        Ld[3 * p + 2] = a2 / fs;
    } else {
        float* o0 = Ls0 + (p * K + (lobe - 1)) * 3;
        float* o1 = Ls1 + (p * K + (lobe - 1)) * 3;
        o0[0] = a0 / fs; o0[1] = a1 / fs; o0[2] = a2 / fs;
        o1[0] = a3 / fs; o1[1] = a4 / fs; o1[2] = a5 / fs;
    }
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct RfLayout {
    RfState st;
    size_t bytes;
};

RfLayout carve_refine(void* base, int64_t P, int waves) {
    Carver c{static_cast<char*>(base), 0};
    RfLayout L;
    L.st.org = c.take<float4>(P);
    L.st.dir = c.take<float4>(2 * P);
    L.st.hit = c.take<int4>(2 * P);
    L.st.bp = c.take<float4>(P);
    L.st.lw = c.take<float4>(P);
    L.st.c0 = c.take<float4>(P);
    L.st.c1 = c.take<float4>(P);
    L.st.sw = c.take<float4>(P);
    L.st.act[0] = c.take<uint32_t>(P);
    L.st.act[1] = c.take<uint32_t>(P);
    L.st.tq[0] = c.take<uint32_t>(2 * P);
    L.st.tq[1] = c.take<uint32_t>(2 * P);
    L.st.cnt = c.take<uint32_t>(4 * (size_t)(waves + 1));
    L.bytes = (c.off + 255) & ~size_t(255);
    return L;
}

// Samples per point and points per chunk; false if one point's samples
// exceed a chunk.
bool refine_chunking(const fipt_bake_params* prm, int64_t N, int64_t& per_pt, int64_t& pts, int64_t& P) {
    per_pt = (int64_t)prm->spp_diffuse + (int64_t)prm->K * prm->spp_specular;
    if (per_pt > RF_SLOT_CAP) return false;
    pts = RF_SLOT_CAP / per_pt;
    P = (N < pts ? N : pts) * per_pt;
    return true;
}

}  // namespace

extern "C" fipt_status fipt_bake_refine_workspace_size(int64_t N, const fipt_bake_params* prm,
                                                       int32_t max_depth, size_t* bytes) {
    FIPT_REQUIRE(prm && bytes, "params / bytes is NULL");
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 32), "bad point count %lld", (long long)N);
    FIPT_REQUIRE(prm->K >= 1 && prm->K <= FIPT_MAX_K, "K must be in [1, %d]", FIPT_MAX_K);
    FIPT_REQUIRE(prm->spp_diffuse >= 1 && prm->spp_specular >= 1, "spp must be >= 1");
    FIPT_REQUIRE(max_depth >= 0 && max_depth < 4096, "max_depth must be in [0, 4096)");
    int64_t per_pt, pts, P;
    FIPT_REQUIRE(refine_chunking(prm, N, per_pt, pts, P),
                 "spp_diffuse + K * spp_specular = %lld exceeds %lld samples per point", (long long)per_pt,
                 (long long)RF_SLOT_CAP);
    *bytes = N == 0 ? 0 : carve_refine(nullptr, P, max_depth + 1).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_bake_refine(fipt_scene* s, const fipt_query* q, int64_t N,
                                        const fipt_bake_params* prm, float sigma_c, int32_t max_depth,
                                        int32_t mis, float* Ld, float* Ls0, float* Ls1,
                                        float* per_sample, void* workspace, size_t ws_bytes,
                                        fipt_stream stream) {
    FIPT_REQUIRE(s && prm, "scene / params is NULL");
    FIPT_REQUIRE(s->has_materials, "fipt_scene_set_materials must be called before a refinement");
    FIPT_REQUIRE(prm->order == nullptr, "params->order is for fipt_bake only");
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 32), "bad point count %lld", (long long)N);
    FIPT_REQUIRE(prm->K >= 1 && prm->K <= FIPT_MAX_K, "K must be in [1, %d]", FIPT_MAX_K);
    FIPT_REQUIRE(prm->spp_diffuse >= 1 && prm->spp_specular >= 1, "spp must be >= 1");
    FIPT_REQUIRE(max_depth >= 0 && max_depth < 4096, "max_depth must be in [0, 4096)");
    for (int k = 0; k < prm->K; ++k)
        FIPT_REQUIRE(prm->sigma[k] > 0.0f && prm->sigma[k] <= 1.0f, "sigma[%d] not in (0, 1]", k);
    int64_t per_pt, pts, P;
    FIPT_REQUIRE(refine_chunking(prm, N, per_pt, pts, P),
                 "spp_diffuse + K * spp_specular = %lld exceeds %lld samples per point", (long long)per_pt,
                 (long long)RF_SLOT_CAP);
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(q && Ld && Ls0 && Ls1, "NULL query / output array");
    FIPT_REQUIRE(fipt_aligned(q, 8) && fipt_aligned(Ld, 4) && fipt_aligned(Ls0, 4) &&
                 fipt_aligned(Ls1, 4) && fipt_aligned(per_sample, 4), "misaligned array");
    const int waves = max_depth + 1;
    RfLayout lay = carve_refine(nullptr, P, waves);
    FIPT_REQUIRE(workspace && fipt_aligned(workspace, 256), "workspace must be 256-byte aligned");
    if (ws_bytes < lay.bytes)
        return fipt_set_error(FIPT_ERR_WORKSPACE, "refine workspace %zu < %zu bytes", ws_bytes, lay.bytes);
    lay = carve_refine(workspace, P, waves);
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    RefineArgs R;
    R.A.key = make_uint2((uint32_t)prm->seed, (uint32_t)(prm->seed >> 32));
    R.A.request_id = prm->request_id;
    R.A.point_base = prm->point_base;
    R.A.spp_d = prm->spp_diffuse;
    R.A.spp_s = prm->spp_specular;
    R.A.K = prm->K;
    set_strata(R.A);
    for (int k = 0; k < FIPT_MAX_K; ++k) R.A.sigma[k] = k < prm->K ? prm->sigma[k] : 1.0f;
    R.sigma_c = sigma_c;
    R.max_depth = max_depth;
    R.mis = mis != 0;
    R.smax = prm->spp_diffuse > prm->spp_specular ? prm->spp_diffuse : prm->spp_specular;
    R.per_pt = (int)per_pt;
    const bool stats = prm->stats != nullptr;
    int sms = 0, occ = 0;
    FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->ctx->device));
    FIPT_CUDA(stats ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rf_trace<true>, RF_TRACE_THREADS, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_rf_trace<false>, RF_TRACE_THREADS, 0));
    const unsigned trace_grid = (unsigned)(sms * (occ > 0 ? occ : 1));
    const unsigned shade_grid = (unsigned)(sms * 8);
    const SceneView sv = s->view();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int64_t p0 = 0; p0 < N; p0 += pts) {
        RfChunk C;
        C.q = q + p0;
        C.p0 = p0;
        C.n_pts = N - p0 < pts ? N - p0 : pts;
        C.P = C.n_pts * per_pt;
        FIPT_CUDA(cudaMemsetAsync(lay.st.cnt, 0, sizeof(uint32_t) * 4 * (size_t)(waves + 1), st));
        const unsigned gen_grid = blocks(C.P, RF_SHADE_THREADS) < shade_grid ? blocks(C.P, RF_SHADE_THREADS) : shade_grid;
        FIPT_LAUNCH(k_rf_gen, gen_grid, RF_SHADE_THREADS, 0, st, sv, C, R, lay.st);
        for (int w = 0; w < waves; ++w) {
            if (w >= 16 && (w & 15) == 0) {    // deep limits: stop once no ray is queued
                uint32_t queued = 0;
                FIPT_CUDA(cudaMemcpyAsync(&queued, lay.st.cnt + 4 * w, sizeof(queued), cudaMemcpyDeviceToHost, st));
                FIPT_CUDA(cudaStreamSynchronize(st));
                if (queued == 0) break;
            }
            if (stats)
                FIPT_LAUNCH(k_rf_trace<true>, trace_grid, RF_TRACE_THREADS, 0, st, sv, lay.st, w,
                            s->ctx->status, prm->stats);
            else
                FIPT_LAUNCH(k_rf_trace<false>, trace_grid, RF_TRACE_THREADS, 0, st, sv, lay.st, w,
                            s->ctx->status, nullptr);
            FIPT_LAUNCH(k_rf_shade, shade_grid, RF_SHADE_THREADS, 0, st, sv, C, R, lay.st, w);
        }
        const unsigned red_grid = blocks(C.n_pts * (1 + prm->K), RF_SHADE_THREADS);
        if (per_sample)
            FIPT_LAUNCH(k_rf_reduce<true>, red_grid, RF_SHADE_THREADS, 0, st, C, R, lay.st, Ld, Ls0, Ls1,
                        per_sample);
        else
            FIPT_LAUNCH(k_rf_reduce<false>, red_grid, RF_SHADE_THREADS, 0, st, C, R, lay.st, Ld, Ls0, Ls1,
                        nullptr);
    }
    FIPT_LAUNCHED("bake_refine");
    return FIPT_OK;
}
