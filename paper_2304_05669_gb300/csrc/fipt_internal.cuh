// Internal declarations shared by the CUDA translation units of libfipt.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

#include "../../include/fipt.h"

// ---------------------------------------------------------------- host glue
struct fipt_ctx {
    int device;
    int32_t* status;    // device status word (FIPT_DEV_* bits)
};

// Device-resident scene constants, written by the build kernels.
struct SceneConst {
    int lo_key[3];      // vertex bounding box as order-preserving ints
    int hi_key[3];
    float lo[3];
    float hi[3];
    float eps;          // ray-origin offset, 1e-4 * largest extent
    int n_emit;         // emitter triangles (any L_e channel > 0)
    double A_emit;      // their total area
};

// Internal BVH node (64 bytes): both child boxes plus child references.
// A reference >= 0 is an internal node; < 0 is the leaf ~ref (one triangle
// at that sorted position).
//   a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//   b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//   c = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//   d = (child0, child1, -, -)
struct __align__(16) BvhNode {
    float4 a, b, c;
    int4 d;
};

struct SceneView {
    const BvhNode* nodes;   // max(T-1, 1)
    const float4* tris;     // 3 per leaf: (v0, orig id bits), (v1, 0), (v2, 0)
    const float4* shade;    // 2 per leaf: (Le rgb, 0), (cache rgb, 0)
    const SceneConst* cst;
    int64_t T;
    int n_inner;            // internal nodes: a reference r is valid iff -T <= r < n_inner
    int max_steps;          // node + leaf visits a valid tree can need for one ray (2T + 2)
    const float4* mats;     // 2 per leaf: (albedo rgb, roughness), (metallic, 0, 0, 0)
    const int32_t* emit_leaf;   // emitter triangles in original index order -> leaf
    const double* emit_cdf;     // cumulative emitter areas (same order)
    const float* env;           // environment radiance [H][W][3] for misses, or NULL
    int env_w, env_h;
    const float4* vox;          // voxel radiance cache [R^3] (mean rgb, count), or NULL
    int vox_r;
};

struct fipt_scene {
    fipt_ctx* ctx;
    int64_t nV, T;
    SceneConst* cst;
    BvhNode* nodes;
    float4* tris;
    float4* shade;
    int32_t* order;        // [T] original index at each sorted position
    uint64_t* keys;        // [T] sorted Morton codes
    int32_t* range;        // [(T-1)*3] first, last, split
    int32_t* parent;       // [T-1]
    int32_t* leaf_parent;  // [T]
    int32_t* flags;        // [T-1]
    uint64_t* keys_alt;
    uint32_t* vals;
    uint32_t* vals_alt;
    uint32_t* hist;
    float4* mats;          // [2T] per-leaf materials (fipt_scene_set_materials)
    int32_t* inv;          // [T] leaf of each original triangle
    int32_t* emit_leaf;    // [T] (first n_emit used)
    double* emit_cdf;      // [T]
    bool has_materials = false;
    bool restructured = false;    // fipt_scene_optimize / relayout ran (range[] is the radix tree's only)
    BvhNode* nodes_alt = nullptr; // second node array (relayout target)
    int32_t* scratch = nullptr;   // [3 (T-1)] relayout scratch
    const float* env = nullptr;   // caller-owned environment map
    int env_w = 0, env_h = 0;
    const float4* vox = nullptr;  // caller-owned voxel radiance cache
    int vox_r = 0;
    size_t ws_bytes;
    SceneView view() const {
        const int64_t steps = 2 * T + 2;
        return SceneView{nodes, tris, shade, cst, T, (int)(T > 1 ? T - 1 : 1),
                         (int)(steps < 2147483647 ? steps : 2147483647), mats, emit_leaf, emit_cdf,
                         env, env_w, env_h, vox, vox_r};
    }
};

// Bake parameters as the kernels read them.
struct BakeArgs {
    uint2 key;
    uint32_t request_id;
    uint32_t point_base;
    int spp_d, spp_s, K;
    int nx_d, nx_s;          // strata along u1 of the diffuse / specular samples (see strat_cols)
    float sigma[FIPT_MAX_K];
};

// Jittered strata of a (point, lobe) pair's S lobe samples: an nx x ny grid
// over the sampling uniforms (u1, u2), nx the largest divisor of S with
// nx^2 <= S, ny = S / nx; sample s lies in cell (s mod nx, s div nx).
inline int strat_cols(int S) {
    int nx = 1;
    for (int d = 1; (int64_t)d * d <= S; ++d)
        if (S % d == 0) nx = d;
    return nx;
}
inline void set_strata(BakeArgs& A) {
    A.nx_d = strat_cols(A.spp_d);
    A.nx_s = strat_cols(A.spp_s);
}

// Sample s of S in its stratum: u1 = (s mod nx + r1)/nx, u2 = (s div nx +
// r2)/ny, each one IEEE float32 addition and division (round to nearest)
// capped below 1, so the FP64 oracle, forming them the same way, gets the
// same bits.
__device__ __forceinline__ void strat_uv(uint32_t s, int S, int nx, float& u1, float& u2) {
    const uint32_t j = s / (uint32_t)nx, i = s - j * (uint32_t)nx;
    const int ny = S / nx;
    u1 = fminf(__fdiv_rn(__fadd_rn((float)i, u1), (float)nx), 0x1.fffffep-1f);
    u2 = fminf(__fdiv_rn(__fadd_rn((float)j, u2), (float)ny), 0x1.fffffep-1f);
}

// A slice of one request's points for the server's resident bake loop.
// 256-byte aligned and sized: a descriptor never shares a cache line with
// another, so the resident loop can read a published descriptor through L1
// without meeting a line cached before that descriptor was written.
struct alignas(256) BakeChunk {
    SceneView sc;
    const fipt_query* q;     // the chunk's first query (the request's first, with an order)
    float *Ld, *Ls0, *Ls1;   // the chunk's first output rows (the request's first, with an order)
    const int32_t* order;    // NULL, or the chunk's slots of the request's order: slot p bakes query order[p]
    int64_t n;               // points in the chunk
    int64_t warp_begin;      // first global warp of the chunk
    BakeArgs A;              // A.point_base = request-local index of the first point
};

// Host-mapped control block of the server's resident bake loop.
struct ServeShared {
    long long taken;       // one past a recently taken warp item (device: relaxed store; the host's estimate)
    int stop;              // nonzero: every bake-loop warp leaves after the item it holds
    int stop_r;            // nonzero: every render-loop warp leaves after its item
};

// A render request for the server's resident loop (Eq. 5, 8, 14 and the
// loss gradient over rows [0, n) of its slice), in RENDER_ITEM_ROWS-row
// warp items.  256-byte slots, like BakeChunk.
constexpr int FIPT_RENDER_ITEM_ROWS = 512;
struct alignas(256) RenderChunk {
    const float *Ld, *Ls0, *Ls1;                 // the request's table rows
    const float *albedo, *rough, *metal, *Lgt;   // its inputs (device copies)
    float *Lr, *g_albedo, *g_rough, *g_metal;    // its outputs
    double* partial;                             // [ceil(n / 128)] loss partials
    double* loss;
    int64_t n;                                   // rows
    int64_t item_begin;                          // first render item of the chunk
    int K;
    float grid[FIPT_MAX_K];
};

// Device counters of the resident loops.  `pub` and `pub_r` are written only
// by the host's copy stream, each after the descriptors it covers (stream
// order): (published items << FIPT_PUB_CHUNK_BITS) | published descriptors,
// for bake and render items.
constexpr int FIPT_PUB_CHUNK_BITS = 17;
struct ServeCounters {
    unsigned long long head;   // bake items handed out
    long long pub;             // what is published of the bake queue (see above)
    unsigned long long head_r; // render items handed out
    long long pub_r;           // what is published of the render queue
    int take_in;               // orphans of the previous launch taken
    int n_in;                  // orphans of the previous launch
    int n_out;                 // orphans this launch leaves
    int quit;                  // nonzero: a bake warp gave up waiting; the whole bake launch leaves
    int quit_r;                // nonzero: a render warp found no work for long; the render launch leaves
    int pad;
};

// The server's resident bake loop (see k_serve_bake) and render loop (see
// k_serve_render).
fipt_status launch_serve_bake(const BakeChunk* d_chunks, ServeShared* sh, ServeCounters* ctr,
                              const long long* orphan_in, long long* orphan_out, int32_t* done_count,
                              int32_t* done_flag, int32_t* status, int wait_polls, int blocks_per_sm,
                              cudaStream_t st, int flags);
fipt_status launch_serve_render(const RenderChunk* d_rchunks, ServeShared* sh, ServeCounters* ctr, int32_t* rdone,
                                int32_t* rflag, int wait_polls, int blocks_per_sm, cudaStream_t st);
// Blocks of the loops that fit on one SM (the least over their kernels,
// all of 64 threads; loads them too).
fipt_status serve_loop_blocks_per_sm(int* blocks);
int serve_loop_warps(int blocks_per_sm);


fipt_status fipt_set_error(fipt_status s, const char* fmt, ...);
void fipt_count_launch();

// Launches a kernel and counts it (fipt_launch_count reports the total).
#define FIPT_LAUNCH(kern, grid, block, smem, st, ...)          \
    do {                                                       \
        kern<<<(grid), (block), (smem), (st)>>>(__VA_ARGS__);  \
        fipt_count_launch();                                   \
    } while (0)
fipt_status fipt_check_cuda(cudaError_t e, const char* what);
bool fipt_aligned(const void* p, size_t a);

#define FIPT_REQUIRE(cond, ...)                                               \
    do {                                                                       \
        if (!(cond)) return fipt_set_error(FIPT_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

#define FIPT_CUDA(call)                                                 \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return fipt_check_cuda(e_, #call);       \
    } while (0)

#define FIPT_LAUNCHED(what)                                             \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return fipt_check_cuda(e_, what);        \
    } while (0)

// Carves aligned sub-buffers out of a caller workspace.
struct Carver {
    char* base;
    size_t off;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort of (key, value) pairs, 8 bits per pass, in caller
// scratch.  Sorts bits [0, bits) of the keys; returns in *out_keys/out_vals
// which of the two buffers holds the result.  With n_dev (a device count
// <= n) only the first *n_dev keys take part, without a host round trip;
// the buffers past them are left undefined.
size_t radix_sort_scratch_bytes(int64_t n);
// Rebuilds the emitter table (leaves, FP64 area CDF, n_emit, A_emit) from
// the packed triangles and their current L_e.
fipt_status rebuild_emitter_table(fipt_scene* s, cudaStream_t st);
template <class K>
fipt_status radix_sort_pairs(K* keys, K* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                             uint32_t* hist, int64_t n, int bits, cudaStream_t st,
                             K** out_keys, uint32_t** out_vals, const uint32_t* n_dev = nullptr);

// ---------------------------------------------------------------- device math
#define FIPT_DONE (-2147483647 - 1)   // traversal finished (not a node, not a leaf)

__device__ __forceinline__ int float_to_ordered(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ordered_to_float(int i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float u24f(uint32_t w) {
    return (float)(w >> 8) * (1.0f / 16777216.0f);
}

// Ray in the form the watertight test wants (Woop, Benthin, Wald 2013):
// kz = dominant axis of d, kx/ky the others (swapped when d[kz] < 0 to keep
// the winding), shear S.
struct TraceRay {
    float ox, oy, oz;
    float ix, iy, iz;       // 1/d for the slab tests
    float Sx, Sy, Sz;
    int k;                  // kx | ky << 2 | kz << 4
};

__device__ __forceinline__ float pick3(float x, float y, float z, int k) {
    return k == 0 ? x : (k == 1 ? y : z);
}

__device__ __forceinline__ TraceRay make_ray(float ox, float oy, float oz, float dx, float dy,
                                             float dz) {
    TraceRay r;
    r.ox = ox; r.oy = oy; r.oz = oz;
    const float tiny = 1e-20f;
    r.ix = 1.0f / (fabsf(dx) < tiny ? copysignf(tiny, dx) : dx);
    r.iy = 1.0f / (fabsf(dy) < tiny ? copysignf(tiny, dy) : dy);
    r.iz = 1.0f / (fabsf(dz) < tiny ? copysignf(tiny, dz) : dz);
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    int kz = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = pick3(dx, dy, dz, kz);
    if (dkz < 0.0f) { int t = kx; kx = ky; ky = t; }
    r.Sx = pick3(dx, dy, dz, kx) / dkz;
    r.Sy = pick3(dx, dy, dz, ky) / dkz;
    r.Sz = 1.0f / dkz;
    r.k = kx | (ky << 2) | (kz << 4);
    return r;
}

// Watertight ray-triangle test.  Edge functions are computed with separately
// rounded products so that the two triangles sharing an edge get exactly
// opposite values; exact zeros are recomputed in double.  Returns the hit
// distance in *t (t > 0) and the facing (front: d . n_g < 0, i.e. det > 0).
__device__ __forceinline__ bool tri_intersect(const TraceRay& r, float4 p0, float4 p1, float4 p2,
                                              float& t, bool& front) {
    const int kx = r.k & 3, ky = (r.k >> 2) & 3, kz = (r.k >> 4) & 3;
    const float Ax0 = p0.x - r.ox, Ay0 = p0.y - r.oy, Az0 = p0.z - r.oz;
    const float Bx0 = p1.x - r.ox, By0 = p1.y - r.oy, Bz0 = p1.z - r.oz;
    const float Cx0 = p2.x - r.ox, Cy0 = p2.y - r.oy, Cz0 = p2.z - r.oz;
    const float Akz = pick3(Ax0, Ay0, Az0, kz), Bkz = pick3(Bx0, By0, Bz0, kz),
                Ckz = pick3(Cx0, Cy0, Cz0, kz);
    const float Ax = fmaf(-r.Sx, Akz, pick3(Ax0, Ay0, Az0, kx));
    const float Ay = fmaf(-r.Sy, Akz, pick3(Ax0, Ay0, Az0, ky));
    const float Bx = fmaf(-r.Sx, Bkz, pick3(Bx0, By0, Bz0, kx));
    const float By = fmaf(-r.Sy, Bkz, pick3(Bx0, By0, Bz0, ky));
    const float Cx = fmaf(-r.Sx, Ckz, pick3(Cx0, Cy0, Cz0, kx));
    const float Cy = fmaf(-r.Sy, Ckz, pick3(Cx0, Cy0, Cz0, ky));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)__dsub_rn(__dmul_rn((double)Cx, (double)By), __dmul_rn((double)Cy, (double)Bx));
        V = (float)__dsub_rn(__dmul_rn((double)Ax, (double)Cy), __dmul_rn((double)Ay, (double)Cx));
        W = (float)__dsub_rn(__dmul_rn((double)Bx, (double)Ay), __dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    t = __fdiv_rn(T, det);
    front = det > 0.0f;
    return t > 0.0f;
}

// Slab test of both child boxes of a node against [0, tmax], widened by a
// few ulps for the rounding of the slab test itself.  The triangle test can
// round a grazing ray's hit distance further below the box's entry (its
// distance sums vertex offsets that cancel; up to about 1e-4 of it), so a
// box may be culled while it holds a triangle whose float32 distance is
// just below tmax: then another triangle's hit within that gap is kept.
__device__ __forceinline__ void node_test(const TraceRay& r, const BvhNode& n, float tmax,
                                          bool& hit0, bool& hit1, float& t0, float& t1) {
    const float ox = r.ox, oy = r.oy, oz = r.oz;
    const float a0 = (n.a.x - ox) * r.ix, a1 = (n.a.y - ox) * r.ix;
    const float a2 = (n.a.z - oy) * r.iy, a3 = (n.a.w - oy) * r.iy;
    const float a4 = (n.c.x - oz) * r.iz, a5 = (n.c.y - oz) * r.iz;
    const float b0 = (n.b.x - ox) * r.ix, b1 = (n.b.y - ox) * r.ix;
    const float b2 = (n.b.z - oy) * r.iy, b3 = (n.b.w - oy) * r.iy;
    const float b4 = (n.c.z - oz) * r.iz, b5 = (n.c.w - oz) * r.iz;
    const float robust = 1.0000005f;
    const float n0 = fmaxf(fmaxf(fminf(a0, a1), fminf(a2, a3)), fmaxf(fminf(a4, a5), 0.0f));
    const float f0 = fminf(fminf(fmaxf(a0, a1), fmaxf(a2, a3)), fminf(fmaxf(a4, a5), tmax));
    const float n1 = fmaxf(fmaxf(fminf(b0, b1), fminf(b2, b3)), fmaxf(fminf(b4, b5), 0.0f));
    const float f1 = fminf(fminf(fmaxf(b0, b1), fmaxf(b2, b3)), fminf(fmaxf(b4, b5), tmax));
    hit0 = n0 <= f0 * robust;
    hit1 = n1 <= f1 * robust;
    t0 = n0;
    t1 = n1;
}

__device__ __forceinline__ BvhNode load_node(const BvhNode* nodes, int i) {
    const float4* p = reinterpret_cast<const float4*>(nodes + i);
    BvhNode n;
    n.a = __ldg(p + 0);
    n.b = __ldg(p + 1);
    n.c = __ldg(p + 2);
    n.d = __ldg(reinterpret_cast<const int4*>(p + 3));
    return n;
}

// Orthonormal basis (t, b) completing a unit normal n (Duff et al. 2017).
// The branch is taken at n.z >= -1e-6 rather than on the sign of n.z, so a
// face whose normal z is zero (+0, -0 or a rounding-sized value) gets the
// same frame however its normal was rounded.
__device__ __forceinline__ void onb(float nx, float ny, float nz, float3& t, float3& b) {
    const float s = nz >= -1e-6f ? 1.0f : -1.0f;
    const float a = -1.0f / (s + nz);
    const float c = nx * ny * a;
    t = make_float3(1.0f + s * nx * nx * a, s * c, -s * nx);
    b = make_float3(c, s + ny * ny * a, -ny);
}

// Environment radiance for a ray that leaves the scene (unit direction d):
// longitude u = atan2(d.x, -d.z) / 2pi + 1/2, colatitude v = acos(d.y) / pi,
// texel (i, j) centred at ((i + 1/2) / W, (j + 1/2) / H), bilinear with u
// wrapping and v clamped.
__device__ __forceinline__ float3 env_lookup(const SceneView& sc, float dx, float dy, float dz) {
    const int W = sc.env_w, H = sc.env_h;
    const float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
    const float y = fminf(fmaxf(dy * il, -1.0f), 1.0f);
    const float u = atan2f(dx * il, -dz * il) * 0.15915494309189535f + 0.5f;
    const float v = acosf(y) * 0.3183098861837907f;
    const float fx = u * (float)W - 0.5f, fy = v * (float)H - 0.5f;
    const float i0f = floorf(fx), j0f = floorf(fy);
    const float tx = fx - i0f, ty = fy - j0f;
    const int i0 = (int)i0f, j0 = (int)j0f;
    float3 L = make_float3(0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            const int i = ((i0 + di) % W + W) % W;
            const int j = min(max(j0 + dj, 0), H - 1);
            const float w = (di ? tx : 1.0f - tx) * (dj ? ty : 1.0f - ty);
            const float* t = sc.env + 3 * ((size_t)j * W + i);
            L.x += w * __ldg(t);
            L.y += w * __ldg(t + 1);
            L.z += w * __ldg(t + 2);
        }
    return L;
}

// Cache radiance L' at a hit point p: the voxel containing p (cell =
// floor((p - lo) * R / (hi - lo)) per axis, clamped) when a voxel cache is
// set.
__device__ __forceinline__ float3 voxel_lookup(const SceneView& sc, float px, float py, float pz) {
    const SceneConst* c = sc.cst;
    const int R = sc.vox_r;
    const float p[3] = {px, py, pz};
    int ix[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float ext = c->hi[a] - c->lo[a];
        const float f = ext > 0.0f ? (p[a] - c->lo[a]) * ((float)R / ext) : 0.0f;
        ix[a] = min(max((int)floorf(f), 0), R - 1);
    }
    const float4 v = __ldg(sc.vox + ((size_t)ix[2] * R + ix[1]) * R + ix[0]);
    return make_float3(v.x, v.y, v.z);
}

// ---------------------------------------------------------------- traversal
// Traversal stack entries per thread.  k_trace and k_camera keep the stack
// in shared memory (a [depth][thread] column per block); the bake (k_bake,
// k_serve_bake) and the refinement's traversal keep it in a per-thread
// local-memory array.  A ray whose stack would overflow drops the far
// child it could not push (that subtree is not searched) and sets
// FIPT_DEV_STACK_OVERFLOW in the device status word.
#ifndef FIPT_STACK_DEPTH
#define FIPT_STACK_DEPTH 32
#endif
constexpr int STACK_DEPTH = FIPT_STACK_DEPTH;
constexpr float FINF = __builtin_huge_valf();

struct BestHit {
    float t;
    int leaf;
    int orig;
    bool front;
};

// Closest hit of one ray; `stack` is this thread's column of the shared
// stack (element k at stack[k * STRIDE]).  A full stack raises the
// overflow bit (the ray loses that subtree).
template <int STRIDE>
__device__ __forceinline__ void closest_hit(const SceneView& sc, const TraceRay& r, int skip,
                                            int* stack, BestHit& best, int32_t* status) {
    best.t = FINF;
    best.leaf = -1;
    best.orig = 0x7fffffff;
    best.front = false;
    if (sc.T == 0) return;
    int node = 0, sp = 0, steps = 0;
    while (node != FIPT_DONE) {
        while (node >= 0) {
            if (node >= sc.n_inner || ++steps > sc.max_steps) {
                atomicOr(status, node >= sc.n_inner ? FIPT_DEV_BAD_NODE : FIPT_DEV_STEP_LIMIT);
                return;
            }
            const BvhNode n = load_node(sc.nodes, node);
            bool h0, h1;
            float t0, t1;
            node_test(r, n, best.t, h0, h1, t0, t1);
            if (h0 && h1) {
                const bool first0 = t0 <= t1;
                if (sp < STACK_DEPTH) {
                    stack[sp * STRIDE] = first0 ? n.d.y : n.d.x;
                    ++sp;
                } else {
                    atomicOr(status, FIPT_DEV_STACK_OVERFLOW);
                }
                node = first0 ? n.d.x : n.d.y;
            } else if (h0) {
                node = n.d.x;
            } else if (h1) {
                node = n.d.y;
            } else {
                node = sp > 0 ? stack[--sp * STRIDE] : FIPT_DONE;
            }
        }
        while (node < 0 && node != FIPT_DONE) {
            const int leaf = ~node;
            if (leaf >= sc.T || ++steps > sc.max_steps) {
                atomicOr(status, leaf >= sc.T ? FIPT_DEV_BAD_NODE : FIPT_DEV_STEP_LIMIT);
                return;
            }
            const float4 p0 = __ldg(sc.tris + 3 * leaf);
            const int orig = __float_as_int(p0.w);
            if (orig != skip) {
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
            node = sp > 0 ? stack[--sp * STRIDE] : FIPT_DONE;
        }
    }
}

// Counters of an instrumented walk: node visits, triangle tests, deepest
// stack.
struct WalkStats {
    unsigned long long nodes = 0, tris = 0;
    int max_sp = 0;
};

// One round of a warp's speculative walk (Aila and Laine 2009).  Every lane
// descends inner nodes; a lane that reaches a leaf parks it (pleaf) and,
// with SPECULATE, keeps descending until every lane holds a leaf or is
// done; the parked leaves, and leaves that follow them on the stack, are
// then tested.  A lane whose walk is over has node == FIPT_DONE and
// pleaf < 0; lanes without a ray call with that state and just vote.  All
// 32 lanes of the warp must call it together.  `stack` is the lane's
// column of the shared stack (entry k at stack[k * STRIDE]).  A lane with
// stop_on_hit ends its walk at the first triangle that improves `best`.
template <int STRIDE, bool STATS, bool SPECULATE>
__device__ __forceinline__ void warp_walk(const SceneView& sc, const TraceRay& r, int skip, BestHit& best,
                                          int& node, int& pleaf, int& sp, int& steps, int* stack,
                                          int32_t* status, WalkStats& ws, bool stop_on_hit = false) {
    for (;;) {
        if (node >= 0 && (SPECULATE || pleaf < 0)) {
            if (node >= sc.n_inner || ++steps > sc.max_steps) {
                atomicOr(status, node >= sc.n_inner ? FIPT_DEV_BAD_NODE : FIPT_DEV_STEP_LIMIT);
                node = FIPT_DONE;
                pleaf = -1;
                sp = 0;
            } else {
                const BvhNode n = load_node(sc.nodes, node);
                if (STATS) ++ws.nodes;
                bool h0, h1;
                float t0, t1;
                node_test(r, n, best.t, h0, h1, t0, t1);
                if (h0 && h1) {
                    const bool first0 = t0 <= t1;
                    if (sp < STACK_DEPTH) {
                        stack[sp * STRIDE] = first0 ? n.d.y : n.d.x;
                        ++sp;
                        if (STATS) ws.max_sp = max(ws.max_sp, sp);
                    } else {
                        atomicOr(status, FIPT_DEV_STACK_OVERFLOW);
                    }
                    node = first0 ? n.d.x : n.d.y;
                } else if (h0) {
                    node = n.d.x;
                } else if (h1) {
                    node = n.d.y;
                } else {
                    node = sp > 0 ? stack[--sp * STRIDE] : FIPT_DONE;
                }
            }
        }
        if (node < 0 && node != FIPT_DONE && pleaf < 0) {   // park the first leaf found
            pleaf = ~node;
            node = sp > 0 ? stack[--sp * STRIDE] : FIPT_DONE;
        }
        if (!__any_sync(0xffffffffu, pleaf < 0 && node >= 0)) break;   // every lane has a leaf or is done
    }
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
            if (STATS) ++ws.tris;
            const float4 p1 = __ldg(sc.tris + 3 * leaf + 1), p2 = __ldg(sc.tris + 3 * leaf + 2);
            float t;
            bool fr;
            if (tri_intersect(r, p0, p1, p2, t, fr) && (t < best.t || (t == best.t && orig < best.orig))) {
                best.t = t;
                best.leaf = leaf;
                best.orig = orig;
                best.front = fr;
                if (stop_on_hit) {
                    node = FIPT_DONE;
                    sp = 0;
                    break;
                }
            }
        }
        if (node < 0 && node != FIPT_DONE) {      // the next entry is a leaf too
            pleaf = ~node;
            node = sp > 0 ? stack[--sp * STRIDE] : FIPT_DONE;
        }
    }
}

