// Ray traversal kernels: closest hit, pinhole first hits, query compaction
// and the bake of the factorized shading terms (Eq. 6-7, Eq. 9, Sec. 6).
//
// Traversal is a per-thread stack walk of the binary LBVH in "while-while"
// form (inner nodes until a leaf, then leaves until an inner node).  The
// first-hit kernels keep the stack in shared memory, laid out
// [depth][thread] so that the threads of a warp touch consecutive banks;
// the bake keeps it in local memory (see bake_item).  Node (64 B) and
// triangle (48 B) reads are 16-byte vector loads through the read-only
// path.
#include "fipt_internal.cuh"
#include "render_math.cuh"

namespace {

constexpr int TRACE_THREADS = 128;

__global__ void __launch_bounds__(TRACE_THREADS)
k_trace(SceneView sc, const float* __restrict__ orig, const float* __restrict__ dir, int64_t n,
        const int32_t* __restrict__ skip, int32_t* __restrict__ hit_tri, float* __restrict__ hit_t,
        int32_t* __restrict__ hit_front, int32_t* status) {
    __shared__ int stk[STACK_DEPTH * TRACE_THREADS];
    const int64_t i = blockIdx.x * (int64_t)TRACE_THREADS + threadIdx.x;
    if (i >= n) return;
    const TraceRay r = make_ray(orig[3 * i], orig[3 * i + 1], orig[3 * i + 2], dir[3 * i],
                                dir[3 * i + 1], dir[3 * i + 2]);
    BestHit b;
    closest_hit<TRACE_THREADS>(sc, r, skip ? skip[i] : -1, stk + threadIdx.x, b, status);
    hit_tri[i] = b.leaf >= 0 ? b.orig : -1;
    hit_t[i] = b.t;
    hit_front[i] = b.leaf >= 0 && b.front ? 1 : 0;
}

__global__ void __launch_bounds__(TRACE_THREADS)
k_camera(SceneView sc, const float* __restrict__ cams, int W, int H, int64_t P,
         fipt_query* __restrict__ out, int32_t* __restrict__ valid, int32_t* status) {
    __shared__ int stk[STACK_DEPTH * TRACE_THREADS];
    const int64_t p = blockIdx.x * (int64_t)TRACE_THREADS + threadIdx.x;
    if (p >= P) return;
    const int64_t wh = (int64_t)W * H;
    const int v = (int)(p / wh);
    const int64_t rem = p - v * wh;
    const int j = (int)(rem / W), i = (int)(rem - (int64_t)j * W);
    const float* c = cams + 10 * v;
    float fx = c[3], fy = c[4], fz = c[5];
    const float fl = 1.0f / sqrtf(fx * fx + fy * fy + fz * fz);
    fx *= fl; fy *= fl; fz *= fl;
    const float ux = c[6], uy = c[7], uz = c[8];
    float rx = fy * uz - fz * uy, ry = fz * ux - fx * uz, rz = fx * uy - fy * ux;
    const float rl = 1.0f / sqrtf(rx * rx + ry * ry + rz * rz);
    rx *= rl; ry *= rl; rz *= rl;
    const float vx = ry * fz - rz * fy, vy = rz * fx - rx * fz, vz = rx * fy - ry * fx;
    const float th = tanf(0.5f * c[9]);
    const float sx = (2.0f * ((float)i + 0.5f) / (float)W - 1.0f) * th * ((float)W / (float)H);
    const float sy = (1.0f - 2.0f * ((float)j + 0.5f) / (float)H) * th;
    float dx = fx + sx * rx + sy * vx, dy = fy + sx * ry + sy * vy, dz = fz + sx * rz + sy * vz;
    const float dl = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    dx *= dl; dy *= dl; dz *= dl;
    const TraceRay r = make_ray(c[0], c[1], c[2], dx, dy, dz);
    BestHit b;
    closest_hit<TRACE_THREADS>(sc, r, -1, stk + threadIdx.x, b, status);
    fipt_query qr;
    if (b.leaf < 0) {
        for (int a = 0; a < 3; ++a) { qr.x[a] = 0.0f; qr.n[a] = 0.0f; qr.wo[a] = 0.0f; }
        qr.tri = -1;
        valid[p] = 0;
    } else {
        const float4 p0 = __ldg(sc.tris + 3 * b.leaf), p1 = __ldg(sc.tris + 3 * b.leaf + 1),
                     p2 = __ldg(sc.tris + 3 * b.leaf + 2);
        const float e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
        const float e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
        float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
        const float nl = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
        const float sg = (nx * dx + ny * dy + nz * dz) > 0.0f ? -nl : nl;
        qr.x[0] = c[0] + b.t * dx; qr.x[1] = c[1] + b.t * dy; qr.x[2] = c[2] + b.t * dz;
        qr.n[0] = sg * nx; qr.n[1] = sg * ny; qr.n[2] = sg * nz;
        qr.wo[0] = -dx; qr.wo[1] = -dy; qr.wo[2] = -dz;
        qr.tri = b.orig;
        valid[p] = 1;
    }
    out[p] = qr;
}

// ---------------------------------------------------------------- compaction
constexpr int CMP_THREADS = 512;
constexpr int CMP_ITEMS = 8;
constexpr int CMP_TILE = CMP_THREADS * CMP_ITEMS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = warp > 0 ? warp_sums[warp - 1] : 0u;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    return before + x - v;
}

__global__ void __launch_bounds__(CMP_THREADS)
k_count_valid(const int32_t* __restrict__ valid, int64_t P, uint32_t* __restrict__ bsum) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * CMP_TILE + threadIdx.x * CMP_ITEMS;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < CMP_ITEMS; ++k) c += (base + k < P && valid[base + k] != 0) ? 1u : 0u;
    uint32_t tot;
    block_exclusive_scan(c, ws, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_bsum(uint32_t* __restrict__ a, int64_t m, int64_t max_out,
                                                   int64_t* __restrict__ n_out) {
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (int64_t b = 0; b < m; b += 1024) {
        const int64_t i = b + threadIdx.x;
        const uint32_t v = i < m ? a[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(v, ws, &tot);
        if (i < m) a[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = (int64_t)carry < max_out ? (int64_t)carry : max_out;
}

__global__ void __launch_bounds__(CMP_THREADS)
k_compact(const fipt_query* __restrict__ in, const int32_t* __restrict__ valid, int64_t P,
          int64_t max_out, const uint32_t* __restrict__ boff, fipt_query* __restrict__ out,
          int32_t* __restrict__ pixel_of) {
    __shared__ uint32_t ws[32];
    const int64_t base = (int64_t)blockIdx.x * CMP_TILE + threadIdx.x * CMP_ITEMS;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < CMP_ITEMS; ++k) c += (base + k < P && valid[base + k] != 0) ? 1u : 0u;
    uint32_t tot;
    int64_t pos = (int64_t)boff[blockIdx.x] + block_exclusive_scan(c, ws, &tot);
    for (int k = 0; k < CMP_ITEMS; ++k) {
        const int64_t i = base + k;
        if (i < P && valid[i] != 0) {
            if (pos < max_out) {
                out[pos] = in[i];
                if (pixel_of) pixel_of[pos] = (int32_t)i;
            }
            ++pos;
        }
    }
}

// ---------------------------------------------------------------- bake
#ifndef FIPT_BAKE_THREADS
#define FIPT_BAKE_THREADS 64
#endif
#ifndef FIPT_BAKE_MINB
#define FIPT_BAKE_MINB 32        // blocks per SM the register budget must allow (full occupancy, 32 registers)
#endif
constexpr int BAKE_THREADS = FIPT_BAKE_THREADS;


#ifndef FIPT_BAKE_REFILL
#define FIPT_BAKE_REFILL 32      // lanes that must be waiting before a warp draws new rays (32: all that still sample)
#endif
#ifndef FIPT_BAKE_SPECULATE
#define FIPT_BAKE_SPECULATE 1    // keep walking inner nodes while other lanes look for a leaf
#endif

// Bakes one (point, lobe) pair per lane: lobe 0 is the diffuse term, lobe
// k+1 roughness level k.  Each lane walks its pair's samples in order and
// sums their contributions in that order (so the result does not depend on
// scheduling).  All 32 lanes of the warp stay in the loop until every lane
// is done (lanes without a pair, `valid` false, just vote), because three
// warp-level decisions keep the lanes doing the same work at the same time:
//  * refill: a lane whose ray has finished waits until FIPT_BAKE_REFILL
//    lanes (or all remaining lanes) are waiting; they then gather their
//    results and draw their next rays together, so the Philox stream,
//    direction sampling and ray set-up run with many lanes active.  With
//    the default (every lane) the lanes draw the same sample index
//    together, and as the samples are jittered strata of one grid their
//    rays leave through the same cell of directions and walk the tree
//    alike (8 % faster on the building floor than refilling at 28);
//  * speculation (Aila and Laine 2009): a lane that reaches a leaf parks
//    it and keeps descending inner nodes until every lane has a leaf;
//  * leaves are then tested together.
// The traversal stack is a per-thread array in local memory, not a shared
// memory column: the bake then reserves no shared memory and the SM's
// unified L1 / shared storage serves as cache for the nodes and for the
// stack entries actually in use.
// FLAGS: 1 = environment light for misses, 2 = voxel radiance cache (each
// used only where the pair's scene has one, so a launch over chunks of
// several scenes takes the union of their flags).
template <bool STATS, int FLAGS>
__device__ __forceinline__ void bake_item(const SceneView& sc, const fipt_query* __restrict__ q,
                                          const int64_t p, const int lobe, const bool valid,
                                          const BakeArgs& A, float* __restrict__ Ld,
                                          float* __restrict__ Ls0, float* __restrict__ Ls1,
                                          int32_t* status, unsigned long long* stats) {
    constexpr unsigned FULL = 0xffffffffu;
    int stack[STACK_DEPTH];
    float nx = 0.0f, ny = 0.0f, nz = 1.0f, wox = 0.0f, woy = 0.0f, woz = 1.0f;
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    int skip = -1;
    if (valid) {
        const float2* qp = reinterpret_cast<const float2*>(q + p);
        const float2 q0 = qp[0], q1 = qp[1], q2 = qp[2], q3 = qp[3], q4 = qp[4];
        px = q0.x; py = q0.y; pz = q1.x;
        nx = q1.y; ny = q2.x; nz = q2.y;
        wox = q3.x; woy = q3.y; woz = q4.x;
        skip = __float_as_int(q4.y);
        const float il = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
        nx *= il; ny *= il; nz *= il;
        const float jl = 1.0f / sqrtf(wox * wox + woy * woy + woz * woz);
        wox *= jl; woy *= jl; woz *= jl;
    }
    const float mu_o = nx * wox + ny * woy + nz * woz;
    const int K = A.K;
    // pairs with nothing to sample: padding lanes, and specular terms of
    // points seen at grazing angles (defined as zero)
    const bool grazing = lobe > 0 && mu_o <= 1e-2f;
    const int S = (!valid || grazing) ? 0 : (lobe == 0 ? A.spp_d : A.spp_s);
    float a2 = 0.0f, g1o = 0.0f;
    if (lobe > 0) {
        float sg = A.sigma[0];
#pragma unroll
        for (int k = 1; k < FIPT_MAX_K; ++k)
            if (lobe - 1 == k) sg = A.sigma[k];
        const float al = sg * sg;
        a2 = al * al;
        g1o = 2.0f * mu_o / (mu_o + sqrtf(a2 + (1.0f - a2) * mu_o * mu_o));
    }
    float3 tb, bb;
    onb(nx, ny, nz, tb, bb);
    const float eps = sc.cst->eps;
    const float ox = px + eps * nx, oy = py + eps * ny, oz = pz + eps * nz;
    const uint32_t pid = A.point_base + (uint32_t)p;

    float acc0x = 0, acc0y = 0, acc0z = 0, acc1x = 0, acc1y = 0, acc1z = 0;
    float wF0 = 1.0f, wF1 = 0.0f;
    float rdx = 0.0f, rdy = 0.0f, rdz = 1.0f;     // current ray direction (environment lookups)
    int s = 0, node = FIPT_DONE, pleaf = -1, sp = 0, steps = 0;
    bool active = false;
    TraceRay r;
    BestHit best;
    best.leaf = -1;
    unsigned long long n_rays = 0, n_nodes = 0, n_tris = 0;
    int max_sp = 0;

    for (;;) {
        // ---------------- refill: gather finished rays, draw new ones together
        const bool idle = node == FIPT_DONE && pleaf < 0;
        const bool need = idle && (active || s < S);
        const unsigned m_need = __ballot_sync(FULL, need);
        const unsigned m_busy = __ballot_sync(FULL, !idle);
        if ((m_need | m_busy) == 0) break;
        if (m_need != 0 && (m_busy == 0 || __popc(m_need) >= FIPT_BAKE_REFILL) && need) {
            if (active) {
                bool lit = best.leaf >= 0;
                float lx = 0.0f, ly = 0.0f, lz = 0.0f;
                if (lit) {
                    const float4 le = __ldg(sc.shade + 2 * best.leaf);
                    float3 ca;
                    if ((FLAGS & 2) && sc.vox) {
                        ca = voxel_lookup(sc, ox + best.t * rdx, oy + best.t * rdy, oz + best.t * rdz);
                    } else {
                        const float4 c4 = __ldg(sc.shade + 2 * best.leaf + 1);
                        ca = make_float3(c4.x, c4.y, c4.z);
                    }
                    lx = (best.front ? le.x : 0.0f) + ca.x;
                    ly = (best.front ? le.y : 0.0f) + ca.y;
                    lz = (best.front ? le.z : 0.0f) + ca.z;
                } else if ((FLAGS & 1) && sc.env) {
                    const float3 e = env_lookup(sc, rdx, rdy, rdz);
                    lx = e.x; ly = e.y; lz = e.z;
                    lit = true;
                }
                if (lit) {
                    if (lobe == 0) {
                        acc0x += lx; acc0y += ly; acc0z += lz;
                    } else {
                        acc0x += lx * wF0; acc0y += ly * wF0; acc0z += lz * wF0;
                        acc1x += lx * wF1; acc1y += ly * wF1; acc1z += lz * wF1;
                    }
                }
                active = false;
            }
            while (s < S) {
                const uint4 rnd = philox4x32_10(make_uint4(pid, (uint32_t)s, (uint32_t)lobe, A.request_id), A.key);
                float u1 = u24f(rnd.x), u2 = u24f(rnd.y);
                strat_uv((uint32_t)s, S, lobe == 0 ? A.nx_d : A.nx_s, u1, u2);
                ++s;
                float sn, cs;
                sincospif(2.0f * u2, &sn, &cs);
                float dx, dy, dz;
                if (lobe == 0) {
                    const float rr = sqrtf(u1), lz = sqrtf(1.0f - u1);
                    const float lx = rr * cs, ly = rr * sn;
                    dx = lx * tb.x + ly * bb.x + lz * nx;
                    dy = lx * tb.y + ly * bb.y + lz * ny;
                    dz = lx * tb.z + ly * bb.z + lz * nz;
                } else {
                    const float om = 1.0f - u1;
                    const float den = om + a2 * u1;
                    const float ch = sqrtf(om / den), sh = sqrtf(a2 * u1 / den);
                    const float lx = sh * cs, ly = sh * sn;
                    const float hx = lx * tb.x + ly * bb.x + ch * nx;
                    const float hy = lx * tb.y + ly * bb.y + ch * ny;
                    const float hz = lx * tb.z + ly * bb.z + ch * nz;
                    const float c = wox * hx + woy * hy + woz * hz;
                    dx = 2.0f * c * hx - wox;
                    dy = 2.0f * c * hy - woy;
                    dz = 2.0f * c * hz - woz;
                    const float mu_i = nx * dx + ny * dy + nz * dz;
                    // a zero sample: the lane traces nothing this round rather than
                    // draw its next sample now, so it stays on the warp's sample index
                    // (and direction cell); +10 % on the building floor
                    if (mu_i <= 0.0f || c <= 0.0f) break;
                    const float g1i = 2.0f * mu_i / (mu_i + sqrtf(a2 + (1.0f - a2) * mu_i * mu_i));
                    const float wt = g1i * g1o * c / (mu_o * ch);
                    const float x1 = 1.0f - c, x2 = x1 * x1;
                    const float F1 = x2 * x2 * x1;
                    wF0 = (1.0f - F1) * wt;
                    wF1 = F1 * wt;
                }
                r = make_ray(ox, oy, oz, dx, dy, dz);
                if (FLAGS) { rdx = dx; rdy = dy; rdz = dz; }
                best.t = FINF;
                best.leaf = -1;
                best.orig = 0x7fffffff;
                best.front = false;
                sp = 0;
                steps = 0;
                node = sc.T > 0 ? 0 : FIPT_DONE;
                active = true;
                if (STATS) ++n_rays;
                break;
            }
        }
        // ---------------- inner nodes (speculative)
        // (the same walk as warp_walk in fipt_internal.cuh, written out here:
        // calling warp_walk from this kernel changes its register allocation
        // and measured 3.8 % slower, with bit-identical results)
        for (;;) {
            if (node >= 0 && (FIPT_BAKE_SPECULATE || pleaf < 0)) {
                if (node >= sc.n_inner || ++steps > sc.max_steps) {
                    atomicOr(status, node >= sc.n_inner ? FIPT_DEV_BAD_NODE : FIPT_DEV_STEP_LIMIT);
                    node = FIPT_DONE;
                    pleaf = -1;
                    sp = 0;
                } else {
                    const BvhNode n = load_node(sc.nodes, node);
                    if (STATS) ++n_nodes;
                    bool h0, h1;
                    float t0, t1;
                    node_test(r, n, best.t, h0, h1, t0, t1);
                    if (h0 && h1) {
                        const bool first0 = t0 <= t1;
                        if (sp < STACK_DEPTH) {
                            stack[sp] = first0 ? n.d.y : n.d.x;
                            ++sp;
                            if (STATS) max_sp = max(max_sp, sp);
                        } else {
                            atomicOr(status, FIPT_DEV_STACK_OVERFLOW);
                        }
                        node = first0 ? n.d.x : n.d.y;
                    } else if (h0) {
                        node = n.d.x;
                    } else if (h1) {
                        node = n.d.y;
                    } else {
                        node = sp > 0 ? stack[--sp] : FIPT_DONE;
                    }
                }
            }
            if (node < 0 && node != FIPT_DONE && pleaf < 0) {   // park the first leaf found
                pleaf = ~node;
                node = sp > 0 ? stack[--sp] : FIPT_DONE;
            }
            if (!__any_sync(FULL, pleaf < 0 && node >= 0)) break;   // every lane has a leaf or is done
        }
        // ---------------- leaves
        while (pleaf >= 0) {
            const int leaf = pleaf;
            pleaf = -1;
            if (leaf >= sc.T || ++steps > sc.max_steps) {
                atomicOr(status, leaf >= sc.T ? FIPT_DEV_BAD_NODE : FIPT_DEV_STEP_LIMIT);
                node = FIPT_DONE;
                sp = 0;
                break;
            }
            const float4 p0 = __ldg(sc.tris + 3 * leaf);
            const int orig = __float_as_int(p0.w);
            if (orig != skip) {
                if (STATS) ++n_tris;
                const float4 p1 = __ldg(sc.tris + 3 * leaf + 1), p2 = __ldg(sc.tris + 3 * leaf + 2);
                float t;
                bool fr;
                if (tri_intersect(r, p0, p1, p2, t, fr) &&
                    (t < best.t || (t == best.t && orig < best.orig))) {
                    best.t = t;
                    best.leaf = leaf;
                    best.orig = orig;
                    best.front = fr;
                }
            }
            if (node < 0 && node != FIPT_DONE) {      // the next entry is a leaf too
                pleaf = ~node;
                node = sp > 0 ? stack[--sp] : FIPT_DONE;
            }
        }
    }

    if (valid) {
        const float fs = (float)(S > 0 ? S : 1);
        if (lobe == 0) {
            Ld[3 * p + 0] = acc0x / fs;
            Ld[3 * p + 1] = acc0y / fs;
            Ld[3 * p + 2] = acc0z / fs;
        } else {
            float* o0 = Ls0 + (p * K + (lobe - 1)) * 3;
            float* o1 = Ls1 + (p * K + (lobe - 1)) * 3;
            o0[0] = acc0x / fs; o0[1] = acc0y / fs; o0[2] = acc0z / fs;
            o1[0] = acc1x / fs; o1[1] = acc1y / fs; o1[2] = acc1z / fs;
        }
    }
    if (STATS) {
        atomicAdd(&stats[0], n_rays);
        atomicAdd(&stats[1], n_nodes);
        atomicAdd(&stats[2], n_tris);
        atomicMax(&stats[3], (unsigned long long)max_sp);
    }
}

// A warp holds 32 consecutive points of one lobe; consecutive warps cycle
// through the lobes of the same 32 points.
template <bool STATS, int FLAGS>
__global__ void __launch_bounds__(BAKE_THREADS, FIPT_BAKE_MINB)
k_bake(SceneView sc, const fipt_query* __restrict__ q, int64_t N, BakeArgs A,
       float* __restrict__ Ld, float* __restrict__ Ls0, float* __restrict__ Ls1, int32_t* status,
       unsigned long long* stats, const int32_t* __restrict__ order) {
    const int L = 1 + A.K;
    const int64_t g = blockIdx.x * (int64_t)BAKE_THREADS + threadIdx.x;
    const int64_t w = g >> 5;
    const int lane = (int)(g & 31);
    const int lobe = (int)(w % L);
    const int64_t p = (w / L) * 32 + lane;
    if ((w / L) * 32 >= N) return;          // whole warp past the end
    bool valid = p < N;
    int64_t pq = p;                         // the query this slot bakes
    if (order && valid) {
        pq = order[p];
        if (pq < 0 || pq >= N) {
            atomicOr(status, FIPT_DEV_BAD_INDEX);
            valid = false;
            pq = 0;
        }
    }
    bake_item<STATS, FLAGS>(sc, q, pq, lobe, valid, A, Ld, Ls0, Ls1, status, stats);
}

// ---------------------------------------------------------------- device-resident serving loop
__device__ __forceinline__ long long ld_relaxed_gpu(const long long* p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_acquire_gpu(const long long* p) {
    long long v;
    asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *reinterpret_cast<const volatile int*>(p); }
__device__ __forceinline__ void st_release_sys(int* p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(long long* p, long long v) {
    asm volatile("st.relaxed.sys.global.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Takes the next published render item, if there is one, with a
// compare-and-swap (render items are taken only when published, so no warp
// ever waits on one); *nch = render descriptors published.
__device__ __forceinline__ bool take_render_item(ServeCounters* ctr, long long* w, int* nch) {
    unsigned long long h = (unsigned long long)ld_relaxed_gpu(reinterpret_cast<const long long*>(&ctr->head_r));
    const unsigned long long avail = (unsigned long long)(ld_relaxed_gpu(&ctr->pub_r) >> FIPT_PUB_CHUNK_BITS);
    while (h < avail) {
        const unsigned long long old = atomicCAS(&ctr->head_r, h, h + 1);
        if (old == h) {
            *w = (long long)h;
            *nch = (int)(ld_acquire_gpu(&ctr->pub_r) & ((1 << FIPT_PUB_CHUNK_BITS) - 1));
            return true;
        }
        h = old;
    }
    return false;
}

// One render item: rows [512 i, 512 i + 512) of the request, as four
// blocks of fipt_render::RENDER_BLOCK rows, each block's loss partial in
// the order the render kernels sum it (the warp stands in for the block's
// four warps one after the other).
__device__ __forceinline__ void render_item(const RenderChunk& RC, int64_t il, int lane) {
    using namespace fipt_render;
    Grid g;
    g.K = RC.K;
#pragma unroll
    for (int k = 0; k < FIPT_MAX_K; ++k) g.s[k] = RC.grid[k];
    const int64_t nb = (RC.n + RENDER_BLOCK - 1) / RENDER_BLOCK;
    constexpr int BLOCKS = FIPT_RENDER_ITEM_ROWS / RENDER_BLOCK;
    for (int vb = 0; vb < BLOCKS; ++vb) {
        const int64_t b = il * BLOCKS + vb;
        if (b >= nb) break;
        double part = 0.0;
        for (int j = 0; j < RENDER_BLOCK / 32; ++j) {
            const int64_t p = b * RENDER_BLOCK + j * 32 + lane;
            float loss = 0.0f;
            if (p < RC.n)
                loss = render_point_fwd_grad(p, g, RC.Ld, RC.Ls0, RC.Ls1, RC.albedo, RC.rough, RC.metal, RC.Lgt,
                                             nullptr, RC.Lr, RC.g_albedo, RC.g_rough, RC.g_metal);
            part += (double)warp_sum_down(loss);
        }
        if (lane == 0) RC.partial[b] = part;
    }
}

// The request's loss from its partials, in the order of the render
// kernels' final sum (RENDER_SUM_THREADS strided sums, a shuffle per warp,
// the warps in order); lane 0 returns it.
__device__ __forceinline__ double render_loss(const RenderChunk& RC, int lane) {
    using namespace fipt_render;
    const int64_t nb = (RC.n + RENDER_BLOCK - 1) / RENDER_BLOCK;
    double t = 0.0;
    for (int j = 0; j < RENDER_SUM_THREADS / 32; ++j) {
        double acc = 0.0;
        for (int64_t i = j * 32 + lane; i < nb; i += RENDER_SUM_THREADS) acc += __ldcg(RC.partial + i);
        t += warp_sum_down(acc);
    }
    return t;
}

// Lane 0 of a bake-loop warp: the warp's next bake item (an orphan of the
// previous launch first, else the next from the counter), waited for until
// it is published -> 1 with *w and *nch (descriptors published), or 0 when
// the warp leaves: the host stopped the launch, or a warp waited
// wait_polls naps without work (it then makes the whole launch leave); a
// leaving warp records its item as an orphan.  Not inlined, so the bake
// walk's register allocation carries none of this.
__device__ __noinline__ int serve_take_bake(ServeShared* sh, ServeCounters* ctr,
                                            const long long* __restrict__ orphan_in,
                                            long long* __restrict__ orphan_out, int wait_polls, long long* w,
                                            int* nch) {
    if (ld_volatile_int(&ctr->quit) || ld_volatile_int(&sh->stop)) return 0;
    long long held;
    const int k = atomicAdd(&ctr->take_in, 1);
    if (k < ctr->n_in) {
        held = __ldcg(orphan_in + k);
    } else {
        held = (long long)atomicAdd(&ctr->head, 1ULL);
        st_relaxed_sys(&sh->taken, held + 1);   // tells the scheduler how far the loop has got
    }
    int idle = 0;
    unsigned nap = 256;
    for (;;) {
        if ((ld_relaxed_gpu(&ctr->pub) >> FIPT_PUB_CHUNK_BITS) > held) {
            *nch = (int)(ld_acquire_gpu(&ctr->pub) & ((1 << FIPT_PUB_CHUNK_BITS) - 1));
            *w = held;
            return 1;
        }
        const bool give_up = ++idle > wait_polls;
        if (give_up) atomicExch(&ctr->quit, 1);
        if (give_up || ld_volatile_int(&ctr->quit) || ((idle & 7) == 0 && ld_volatile_int(&sh->stop))) {
            orphan_out[atomicAdd(&ctr->n_out, 1)] = held;
            return 0;
        }
        __nanosleep(nap);
        if (nap < 32768) nap *= 2;
    }
}

// The server's bake loop: resident warps take bake items (32 points of one
// chunk, one lobe) in publication order from a device counter with one
// atomicAdd each (no compare-and-swap retries, so thousands of warps do not
// serialise on the counter), bake each exactly as k_bake would, and count
// it done; the warp that completes a chunk raises the chunk's flag in
// host-mapped memory, where the server's scheduler sees it without a copy.
// The host publishes work by copying chunk descriptors to `chunks` and
// then the published item and descriptor counts to ctr->pub, in that order
// on one copy stream, so the loop polls device memory (never host memory,
// whose system-scope loads would slow the warps still baking); each warp
// that takes a new item writes how far it got to sh->taken, from which the
// host decides how much more to publish.  A warp whose item is not
// published yet polls with naps growing to 32 microseconds and reads the
// count once more with acquire semantics before it uses the descriptor.
// The launch ends as a whole: when the host sets sh->stop (it has no work
// left, or it failed), or when a warp has waited wait_polls naps in vain
// (the host did not answer) and sets ctr->quit, every warp leaves -- a
// waiting warp at once, recording its item in `orphan_out`, a busy one
// after its item, without taking another.  The next launch takes the
// orphans first (from `orphan_in`), so no item is lost or taken twice, and
// no orphan waits behind warps that keep running.  A descriptor is read
// only after its publication, and no cache line holds parts of two
// descriptors, so L1 never serves one from before it was written.  Render
// requests have a loop of their own (k_serve_render) beside this one: code
// for them in this kernel cost the bake walk 7 % through its register
// allocation.
template <int FLAGS>
__global__ void __launch_bounds__(BAKE_THREADS, FIPT_BAKE_MINB)
k_serve_bake(const BakeChunk* __restrict__ chunks, ServeShared* sh, ServeCounters* ctr,
             const long long* __restrict__ orphan_in, long long* __restrict__ orphan_out,
             int32_t* __restrict__ done_count, int32_t* done_flag, int32_t* status, int wait_polls) {
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(sizeof(BakeChunk) == 256, "one descriptor per pair of cache lines");
    const int lane = threadIdx.x & 31;
    int ci = 0;
    for (;;) {
        int act = 0;
        long long w = -1;
        int nch = 0;
        if (lane == 0) act = serve_take_bake(sh, ctr, orphan_in, orphan_out, wait_polls, &w, &nch);
        act = __shfl_sync(FULL, act, 0);
        w = __shfl_sync(FULL, w, 0);
        nch = __shfl_sync(FULL, nch, 0);
        if (act == 0) return;
        if (w < chunks[ci].warp_begin) ci = 0;              // an orphan from earlier
        while (ci + 1 < nch && chunks[ci + 1].warp_begin <= w) ++ci;
        const BakeChunk& C = chunks[ci];
        const int L = 1 + C.A.K;
        const int64_t wl = w - C.warp_begin;
        const int lobe = (int)(wl % L);
        const int64_t p = (wl / L) * 32 + lane;
        const bool valid = p < C.n;
        const int64_t pq = (C.order && valid) ? (int64_t)C.order[p] : p;
        bake_item<false, FLAGS>(C.sc, C.q, pq, lobe, valid, C.A, C.Ld, C.Ls0, C.Ls1, status, nullptr);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            const int items = (int)(((C.n + 31) / 32) * L);
            if (atomicAdd(done_count + ci, 1) == items - 1) {
                __threadfence_system();
                st_release_sys(done_flag + ci, 1);
            }
        }
    }
}

// The server's render loop, resident beside the bake loop on a few block
// slots per SM: its warps take render items (512 rows of one render
// request) by compare-and-swap as the host publishes them (to `rchunks`,
// then ctr->pub_r, on the copy stream), so a render request starts at once
// whatever the bake loop holds; each item runs k_render_fwd_grad's
// arithmetic and writes its blocks' loss partials, and the warp that
// completes a request sums its loss in the render kernels' order, then
// raises the request's flag in host-mapped memory.  Warps never hold an
// item they cannot run, so they may leave one by one: when the host sets
// sh->stop_r, or after wait_polls naps without a render item (ctr->quit_r
// then tells the others); the host starts the loop again when new render
// work is published.
__global__ void __launch_bounds__(BAKE_THREADS, FIPT_BAKE_MINB)
k_serve_render(const RenderChunk* __restrict__ rchunks, ServeShared* sh, ServeCounters* ctr,
               int32_t* __restrict__ rdone, int32_t* rflag, int wait_polls) {
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(sizeof(RenderChunk) == 256, "one descriptor per pair of cache lines");
    const int lane = threadIdx.x & 31;
    int cr = 0;
    for (;;) {
        int act = 0;
        long long w = -1;
        int nch = 0;
        if (lane == 0) {
            int idle = 0;
            unsigned nap = 256;
            for (;;) {
                if (ld_volatile_int(&ctr->quit_r) || ((idle & 7) == 0 && ld_volatile_int(&sh->stop_r))) break;
                if (take_render_item(ctr, &w, &nch)) {
                    act = 1;
                    break;
                }
                if (++idle > wait_polls) {
                    atomicExch(&ctr->quit_r, 1);
                    break;
                }
                __nanosleep(nap);
                if (nap < 32768) nap *= 2;
            }
        }
        act = __shfl_sync(FULL, act, 0);
        w = __shfl_sync(FULL, w, 0);
        nch = __shfl_sync(FULL, nch, 0);
        if (act == 0) return;
        if (w < rchunks[cr].item_begin) cr = 0;
        while (cr + 1 < nch && rchunks[cr + 1].item_begin <= w) ++cr;
        const RenderChunk& RC = rchunks[cr];
        render_item(RC, w - RC.item_begin, lane);
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence();
            const int items = (int)((RC.n + FIPT_RENDER_ITEM_ROWS - 1) / FIPT_RENDER_ITEM_ROWS);
            last = atomicAdd(rdone + cr, 1) == items - 1;
        }
        last = __shfl_sync(FULL, last, 0);
        if (last) {                                      // every partial is written: the loss
            __threadfence();
            const double loss = render_loss(RC, lane);
            if (lane == 0) {
                *RC.loss = loss;
                __threadfence_system();
                st_release_sys(rflag + cr, 1);
            }
        }
    }
}

// Bit k of a 10-bit value to bit 3k (room for the other two axes).
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Sort keys of the query points: the 30-bit Morton code of each position
// in the scene's bounding box (1024 cells per axis); values = indices.
__global__ void k_query_keys(const fipt_query* __restrict__ q, int64_t N, const SceneConst* __restrict__ cst,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float2* qp = reinterpret_cast<const float2*>(q + i);
    const float2 a = qp[0], b = qp[1];
    const float x[3] = {a.x, a.y, b.x};
    uint32_t key = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float ext = cst->hi[ax] - cst->lo[ax];
        const float u = ext > 0.0f ? (x[ax] - cst->lo[ax]) / ext : 0.0f;
        const float c = fminf(fmaxf(u * 1024.0f, 0.0f), 1023.0f);   // NaN -> 0
        key |= spread3_10((uint32_t)c) << ax;
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key, int64_t n,
                         uint32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" fipt_status fipt_trace_closest(fipt_scene* s, const float* orig, const float* dir,
                                          int64_t nR, const int32_t* skip_tri, int32_t* hit_tri,
                                          float* hit_t, int32_t* hit_front, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(nR >= 0 && nR < ((int64_t)1 << 40), "bad ray count %lld", (long long)nR);
    if (nR == 0) return FIPT_OK;
    FIPT_REQUIRE(orig && dir && hit_tri && hit_t && hit_front, "NULL ray / hit array");
    FIPT_REQUIRE(fipt_aligned(orig, 4) && fipt_aligned(dir, 4) && fipt_aligned(hit_tri, 4) &&
                 fipt_aligned(hit_t, 4) && fipt_aligned(hit_front, 4) && fipt_aligned(skip_tri, 4),
                 "arrays must be 4-byte aligned");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    FIPT_LAUNCH(k_trace, blocks(nR, TRACE_THREADS), TRACE_THREADS, 0, static_cast<cudaStream_t>(stream), s->view(), orig, dir, nR, skip_tri, hit_tri, hit_t, hit_front, s->ctx->status);
    FIPT_LAUNCHED("trace_closest");
    return FIPT_OK;
}

extern "C" fipt_status fipt_camera_queries(fipt_scene* s, const float* cams, int32_t nViews,
                                           int32_t W, int32_t H, fipt_query* out, int32_t* valid,
                                           fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(nViews >= 0 && W >= 0 && H >= 0, "negative camera sizes");
    const int64_t P = (int64_t)nViews * W * H;
    if (P == 0) return FIPT_OK;
    FIPT_REQUIRE(P < ((int64_t)1 << 31), "too many pixels");
    FIPT_REQUIRE(cams && out && valid, "NULL camera / output array");
    FIPT_REQUIRE(fipt_aligned(cams, 4) && fipt_aligned(out, 16) && fipt_aligned(valid, 4),
                 "cams 4-byte, out 16-byte, valid 4-byte alignment required");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    FIPT_LAUNCH(k_camera, blocks(P, TRACE_THREADS), TRACE_THREADS, 0, static_cast<cudaStream_t>(stream), s->view(), cams, W, H, P, out, valid, s->ctx->status);
    FIPT_LAUNCHED("camera_queries");
    return FIPT_OK;
}

extern "C" fipt_status fipt_compact_workspace_size(int64_t P, size_t* bytes) {
    FIPT_REQUIRE(bytes && P >= 0, "bad arguments");
    *bytes = (size_t)(blocks(P, CMP_TILE) + 1) * sizeof(uint32_t) + 256;
    return FIPT_OK;
}

extern "C" fipt_status fipt_compact_queries(const fipt_query* in, const int32_t* valid, int64_t P,
                                            int64_t max_out, fipt_query* out, int32_t* pixel_of,
                                            int64_t* n_out, void* ws, size_t ws_bytes,
                                            fipt_stream stream) {
    FIPT_REQUIRE(P >= 0 && P < ((int64_t)1 << 31) && max_out >= 0, "bad sizes");
    FIPT_REQUIRE(n_out && fipt_aligned(n_out, 8), "n_out NULL or not 8-byte aligned");
    size_t need;
    fipt_compact_workspace_size(P, &need);
    if (ws_bytes < need || !ws)
        return fipt_set_error(FIPT_ERR_WORKSPACE, "compact workspace %zu < %zu", ws_bytes, need);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P == 0) {
        FIPT_CUDA(cudaMemsetAsync(n_out, 0, sizeof(int64_t), st));
        return FIPT_OK;
    }
    FIPT_REQUIRE(in && valid && (out || max_out == 0) && fipt_aligned(in, 16) &&
                 fipt_aligned(out, 16) && fipt_aligned(valid, 4) && fipt_aligned(pixel_of, 4),
                 "NULL or misaligned array");
    const unsigned nb = blocks(P, CMP_TILE);
    uint32_t* bsum = static_cast<uint32_t*>(ws);
    FIPT_LAUNCH(k_count_valid, nb, CMP_THREADS, 0, st, valid, P, bsum);
    FIPT_LAUNCH(k_scan_bsum, 1, 1024, 0, st, bsum, nb, max_out, n_out);
    FIPT_LAUNCH(k_compact, nb, CMP_THREADS, 0, st, in, valid, P, max_out, bsum, out, pixel_of);
    FIPT_LAUNCHED("compact_queries");
    return FIPT_OK;
}

namespace {
struct OrderLayout {
    uint32_t *keys, *keys_alt, *vals_alt, *hist;
    size_t bytes;
};
OrderLayout carve_order(void* ws, int64_t N) {
    Carver c{static_cast<char*>(ws), 0};
    OrderLayout L;
    L.keys = c.take<uint32_t>((size_t)N);
    L.keys_alt = c.take<uint32_t>((size_t)N);
    L.vals_alt = c.take<uint32_t>((size_t)N);
    L.hist = c.take<uint32_t>(radix_sort_scratch_bytes(N) / sizeof(uint32_t) + 1);
    L.bytes = c.off + 256;
    return L;
}
}  // namespace

extern "C" fipt_status fipt_query_order_workspace_size(int64_t N, size_t* bytes) {
    FIPT_REQUIRE(bytes && N >= 0 && N < ((int64_t)1 << 31), "bad point count");
    *bytes = carve_order(nullptr, N).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_query_order(fipt_scene* s, const fipt_query* q, int64_t N, int32_t* order,
                                        void* workspace, size_t ws_bytes, fipt_stream stream) {
    FIPT_REQUIRE(s, "scene is NULL");
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 31), "bad point count %lld", (long long)N);
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(q && order, "NULL query / order array");
    FIPT_REQUIRE(fipt_aligned(q, 8) && fipt_aligned(order, 4), "q must be 8-byte aligned, order 4-byte");
    FIPT_REQUIRE(workspace && fipt_aligned(workspace, 256), "workspace must be 256-byte aligned");
    const OrderLayout need = carve_order(nullptr, N);
    if (ws_bytes < need.bytes)
        return fipt_set_error(FIPT_ERR_WORKSPACE, "query order workspace %zu < %zu bytes", ws_bytes, need.bytes);
    const OrderLayout L = carve_order(workspace, N);
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t* vals = reinterpret_cast<uint32_t*>(order);
    FIPT_LAUNCH(k_query_keys, blocks(N, 256), 256, 0, st, q, N, s->cst, L.keys, vals);
    FIPT_LAUNCHED("query order keys");
    uint32_t *sk = nullptr, *sv = nullptr;
    const fipt_status r = radix_sort_pairs<uint32_t>(L.keys, L.keys_alt, vals, L.vals_alt, L.hist, N, 32, st,
                                                     &sk, &sv);
    if (r != FIPT_OK) return r;
    if (sv != vals) FIPT_CUDA(cudaMemcpyAsync(order, sv, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    return FIPT_OK;
}

extern "C" fipt_status fipt_bake(fipt_scene* s, const fipt_query* q, int64_t N,
                                 const fipt_bake_params* prm, float* Ld, float* Ls0, float* Ls1,
                                 fipt_stream stream) {
    FIPT_REQUIRE(s && prm, "scene / params is NULL");
    FIPT_REQUIRE(N >= 0 && N < ((int64_t)1 << 32), "bad point count %lld", (long long)N);
    FIPT_REQUIRE(prm->K >= 1 && prm->K <= FIPT_MAX_K, "K must be in [1, %d]", FIPT_MAX_K);
    FIPT_REQUIRE(prm->spp_diffuse >= 1 && prm->spp_specular >= 1, "spp must be >= 1");
    for (int k = 0; k < prm->K; ++k)
        FIPT_REQUIRE(prm->sigma[k] > 0.0f && prm->sigma[k] <= 1.0f, "sigma[%d] = %g not in (0, 1]",
                     k, (double)prm->sigma[k]);
    if (N == 0) return FIPT_OK;
    FIPT_REQUIRE(q && Ld && Ls0 && Ls1, "NULL query / output array");
    FIPT_REQUIRE(fipt_aligned(q, 8) && fipt_aligned(Ld, 4) && fipt_aligned(Ls0, 4) &&
                 fipt_aligned(Ls1, 4) && fipt_aligned(prm->stats, 8) && fipt_aligned(prm->order, 4),
                 "q must be 8-byte aligned, outputs and order 4-byte");
    FIPT_CUDA(cudaSetDevice(s->ctx->device));
    BakeArgs A;
    A.key = make_uint2((uint32_t)prm->seed, (uint32_t)(prm->seed >> 32));
    A.request_id = prm->request_id;
    A.point_base = prm->point_base;
    A.spp_d = prm->spp_diffuse;
    A.spp_s = prm->spp_specular;
    A.K = prm->K;
    set_strata(A);
    for (int k = 0; k < FIPT_MAX_K; ++k) A.sigma[k] = k < prm->K ? prm->sigma[k] : 1.0f;
    const int64_t warps = ((N + 31) / 32) * (1 + prm->K);
    const int64_t threads = warps * 32;
    const unsigned nb = blocks(threads, BAKE_THREADS);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int flags = (s->env ? 1 : 0) | (s->vox ? 2 : 0);
    const SceneView sv = s->view();
    unsigned long long* stats = prm->stats;
#define FIPT_BAKE_CASE(ST, FL)                                                                   \
    FIPT_LAUNCH((k_bake<ST, FL>), nb, BAKE_THREADS, 0, st, sv, q, N, A, Ld, Ls0, Ls1, s->ctx->status, \
                stats, prm->order)
    if (stats) {
        switch (flags) {
            case 0: FIPT_BAKE_CASE(true, 0); break;
            case 1: FIPT_BAKE_CASE(true, 1); break;
            case 2: FIPT_BAKE_CASE(true, 2); break;
            default: FIPT_BAKE_CASE(true, 3); break;
        }
    } else {
        switch (flags) {
            case 0: FIPT_BAKE_CASE(false, 0); break;
            case 1: FIPT_BAKE_CASE(false, 1); break;
            case 2: FIPT_BAKE_CASE(false, 2); break;
            default: FIPT_BAKE_CASE(false, 3); break;
        }
    }
#undef FIPT_BAKE_CASE
    FIPT_LAUNCHED("bake");
    return FIPT_OK;
}

extern "C" fipt_status fipt_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n,
                                         uint32_t* out, fipt_stream stream) {
    FIPT_REQUIRE(n >= 0, "negative n");
    if (n == 0) return FIPT_OK;
    FIPT_REQUIRE(ctr && key && out, "NULL array");
    FIPT_LAUNCH(k_philox, blocks(n, 256), 256, 0, static_cast<cudaStream_t>(stream), ctr, key, n, out);
    FIPT_LAUNCHED("philox");
    return FIPT_OK;
}

// Launcher of the server's resident bake loop: blocks_per_sm resident blocks
// on every SM of the current device.
fipt_status launch_serve_bake(const BakeChunk* d_chunks, ServeShared* sh, ServeCounters* ctr,
                              const long long* orphan_in, long long* orphan_out, int32_t* done_count,
                              int32_t* done_flag, int32_t* status, int wait_polls, int blocks_per_sm,
                              cudaStream_t st, int flags) {
    int dev = 0, sms = 0;
    FIPT_CUDA(cudaGetDevice(&dev));
    FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const unsigned nb = (unsigned)(sms * blocks_per_sm);
#define FIPT_SERVE_CASE(FL) \
    FIPT_LAUNCH(k_serve_bake<FL>, nb, BAKE_THREADS, 0, st, d_chunks, sh, ctr, orphan_in, orphan_out, done_count, \
                done_flag, status, wait_polls)
    switch (flags) {
        case 0: FIPT_SERVE_CASE(0); break;
        case 1: FIPT_SERVE_CASE(1); break;
        case 2: FIPT_SERVE_CASE(2); break;
        default: FIPT_SERVE_CASE(3); break;
    }
#undef FIPT_SERVE_CASE
    FIPT_LAUNCHED("serve_bake");
    return FIPT_OK;
}

fipt_status launch_serve_render(const RenderChunk* d_rchunks, ServeShared* sh, ServeCounters* ctr, int32_t* rdone,
                                int32_t* rflag, int wait_polls, int blocks_per_sm, cudaStream_t st) {
    int dev = 0, sms = 0;
    FIPT_CUDA(cudaGetDevice(&dev));
    FIPT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    FIPT_LAUNCH(k_serve_render, (unsigned)(sms * blocks_per_sm), BAKE_THREADS, 0, st, d_rchunks, sh, ctr, rdone,
                rflag, wait_polls);
    FIPT_LAUNCHED("serve_render");
    return FIPT_OK;
}

fipt_status serve_loop_blocks_per_sm(int* blocks) {
    const void* fns[] = {(const void*)k_serve_bake<0>, (const void*)k_serve_bake<1>,
                         (const void*)k_serve_bake<2>, (const void*)k_serve_bake<3>,
                         (const void*)k_serve_render};
    int b = 1 << 30;
    for (const void* f : fns) {
        int occ = 0;
        FIPT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, BAKE_THREADS, 0));
        b = std::min(b, occ);
    }
    *blocks = b;
    return FIPT_OK;
}

// Most warps a launch of the resident loop can have (each leaves at most
// one orphan).
int serve_loop_warps(int blocks_per_sm) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * blocks_per_sm * (BAKE_THREADS / 32);
}
