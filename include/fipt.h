/*
 * fipt.h -- C ABI of the GB300 bake of the factorized shading terms of
 * "Factorized Inverse Path Tracing" (Wu et al., ICCV 2023, arXiv 2304.05669).
 *
 * The paper factors the material out of the rendering integral (Sec. 4.1,
 * Eq. 5-7) so that three shading terms per surface point -- the diffuse
 * shading L_d and the two specular shadings L_s0, L_s1 tabulated over a
 * roughness grid (Eq. 8) -- can be baked once and reused by a cheap
 * factorized render.  This library builds a BVH over a triangle mesh, bakes
 * those terms by BRDF importance sampling with the one-segment cache query
 * of Eq. 9 (Sec. 4.2, Sec. 6 stage 1), renders the factorized model with a
 * tone-mapped loss (Eq. 14) and its gradient, and reduces the rendering
 * error per triangle to locate emitters (Sec. 4.4).
 *
 * Conventions shared by every call:
 *  - Every call returns fipt_status; FIPT_OK is 0.  On failure a message is
 *    kept per host thread and returned by fipt_last_error().
 *  - Array arguments are DEVICE pointers on the context's device, owned by
 *    the caller, contiguous, in the dtype and layout stated; they must be
 *    4-byte aligned, and 16-byte aligned where stated.  Host pointers are
 *    marked "host".  Nothing is allocated on the bake/render path: scratch
 *    comes from caller workspaces sized by the *_workspace_size queries.
 *  - Work is enqueued on the caller's stream and is asynchronous.  A kernel
 *    that detects a bad state (traversal stack overflow) records a code in
 *    the context's device status word instead of faulting; read and clear it
 *    with fipt_sync_status().
 *  - Sizes of 0 are valid and enqueue nothing.
 */
#ifndef FIPT_H
#define FIPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fipt_status {
    FIPT_OK = 0,
    FIPT_ERR_INVALID_ARG = 1,   /* null / misaligned pointer, bad size or parameter */
    FIPT_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    FIPT_ERR_WORKSPACE = 3,     /* the workspace passed is smaller than required */
    FIPT_ERR_BUDGET = 4,        /* a request does not fit the server's memory budget */
    FIPT_ERR_TIMEOUT = 5,       /* a bounded wait ran out */
    FIPT_ERR_DEVICE_CHECK = 6,  /* a kernel recorded a failed check (see fipt_sync_status) */
    FIPT_ERR_NOT_FOUND = 7      /* unknown ticket / handle */
} fipt_status;

/* Device status codes written by kernels (bit flags). */
#define FIPT_DEV_STACK_OVERFLOW 1   /* a traversal stack was full; that ray was cut short */
#define FIPT_DEV_BAD_NODE 2         /* a BVH reference was out of range; that ray was stopped */
#define FIPT_DEV_STEP_LIMIT 4       /* a walk exceeded the steps a valid tree allows; stopped */
#define FIPT_DEV_BAD_INDEX 8        /* an input vertex index was outside [0, nV) (read as 0), or a bake
                                       order entry outside [0, N) (that slot baked nothing) */

typedef void* fipt_stream;               /* a cudaStream_t; NULL = the legacy default stream */
typedef struct fipt_ctx fipt_ctx;
typedef struct fipt_scene fipt_scene;

/* One surface query (40 bytes): the point x, its unit normal n on the side
 * it is seen from, the unit viewing direction wo (n . wo > 0), and the index
 * of the triangle x lies on (-1: none).  Sec. 3 / Eq. 2-4: one per camera
 * ray (x, wo); Sec. 4.1: the shadings are baked per input-view pixel. */
typedef struct fipt_query {
    float x[3];
    float n[3];
    float wo[3];
    int32_t tri;
} fipt_query;

#define FIPT_MAX_K 8

/* Bake parameters (host struct).
 *  seed, request_id, point_base: the Philox4x32-10 stream.  Ray s of lobe l
 *    (0 = diffuse, k+1 = roughness level k) at query i draws its two
 *    uniforms from counter (point_base + i, s, l, request_id) under key
 *    (seed low 32 bits, seed high 32 bits): word >> 8 times 2^-24.  Results
 *    therefore do not depend on how a batch is split or scheduled.
 *  spp_diffuse, spp_specular: samples per point for L_d and for each level
 *    of L_s0/L_s1 (Sec. 6 uses 128 and 64).
 *  K, sigma[K]: roughness levels (Eq. 8), each in (0, 1]; alpha = sigma^2.
 *  stats: NULL, or a device pointer to 4 unsigned 64-bit counters to which
 *    the bake ADDS: rays traced, BVH nodes visited, triangles tested, and
 *    (max, not added) the deepest traversal stack seen. */
typedef struct fipt_bake_params {
    uint64_t seed;
    uint32_t request_id;
    uint32_t point_base;
    int32_t spp_diffuse;
    int32_t spp_specular;
    int32_t K;
    float sigma[FIPT_MAX_K];
    unsigned long long* stats;
    /* fipt_bake only (NULL elsewhere): NULL, or a DEVICE int32 [N]
     * permutation of [0, N) (see fipt_query_order); launch slot p then
     * bakes query order[p].  A point's random numbers and outputs use its
     * own index, so only the grouping of points into warps changes; that
     * grouping sets when a lane's parked triangles lower its culling bound,
     * which could change a hit only where float32 puts two triangles' hit
     * distances within rounding of each other (grazing rays), as for
     * fipt_scene_optimize; none has been observed on the room and floor
     * workloads. */
    const int32_t* order;
} fipt_bake_params;

/* ------------------------------------------------------------ context */
const char* fipt_last_error(void);
const char* fipt_status_string(fipt_status s);
/* Library build tag (string literal, host). */
const char* fipt_version(void);
/* Number of kernels this library has launched in the process (all
 * contexts, all threads); benchmarks difference it around a timed region. */
uint64_t fipt_launch_count(void);

/* Creates a context on CUDA device `device` (allocates its 4-byte device
 * status word; the only allocation outside the server).  *out owned by the
 * caller, released with fipt_ctx_destroy. */
fipt_status fipt_ctx_create(int device, fipt_ctx** out);
fipt_status fipt_ctx_destroy(fipt_ctx* ctx);

/* Waits for `stream`, then reads and clears the device status word.
 * *device_code (host, nullable) receives the FIPT_DEV_* bits.  Returns
 * FIPT_ERR_DEVICE_CHECK when any bit was set. */
fipt_status fipt_sync_status(fipt_ctx* ctx, fipt_stream stream, int32_t* device_code);

/* ------------------------------------------------------------ scene */
/* Bytes of device workspace a scene of nV vertices and T triangles needs
 * (BVH nodes, packed triangles, per-triangle radiance, build scratch). */
fipt_status fipt_scene_workspace_size(int64_t nV, int64_t T, size_t* bytes);

/* Builds the scene on the device, stream-ordered, no host synchronisation.
 *  V [nV,3] f32 positions; F [T,3] i32 vertex indices (each in [0, nV));
 *  Le [T,3] f32 view-independent emission (Sec. 3), seen only from the side
 *  (v1-v0)x(v2-v0) points to; cache [T,3] f32 the diffuse radiance cache L'
 *  at each triangle (Eq. 9; a per-triangle stand-in for Sec. 4.2's voxels).
 *  workspace: >= fipt_scene_workspace_size bytes, 256-byte aligned; the
 *  scene keeps pointers into it (caller keeps it alive until destroy).
 *  V, F, Le, cache may be freed once the stream has passed this call.
 * The BVH is a linear BVH: 63-bit Morton codes of triangle box centres
 * quantised in FP64 against the vertex bounding box, a stable radix sort of
 * (code, index), Karras's binary radix tree over the sorted codes, and a
 * bottom-up refit of the node boxes.  T = 0 gives a scene every ray misses. */
fipt_status fipt_scene_create(fipt_ctx* ctx, const float* V, int64_t nV, const int32_t* F,
                              int64_t T, const float* Le, const float* cache, void* workspace,
                              size_t ws_bytes, fipt_stream stream, fipt_scene** out);

/* Treelet restructuring of the scene's tree (Karras and Aila 2013), in
 * place, `passes` bottom-up passes (0 to 16; 0 does nothing): at every
 * internal node the treelet of up to 7 subtrees reached by expanding the
 * largest-area children is given the topology with the least total
 * surface area of its internal nodes (the SAH cost with one triangle per
 * leaf), if that is strictly cheaper.  Leaves and their boxes stay and
 * walks visit fewer nodes.  The closest hit, the (t, triangle) minimum, does
 * not depend on the tree, except where float32 puts several triangles'
 * hit distances within rounding of one another (a ray along a shared edge;
 * a ray grazing a large triangle, whose distance can round about 1e-4 of
 * itself low): the culling bound then depends on the visit order and
 * another of those equally correct hits may be returned.  The radix-tree ranges of fipt_scene_debug_export
 * no longer describe the tree afterwards.  Not an operation of the paper:
 * a property of the acceleration structure only. */
fipt_status fipt_scene_optimize(fipt_scene* scene, int32_t passes, fipt_stream stream);

/* Renumbers the scene's internal nodes depth-first (root 0, a node's first
 * child right after it, its second child after the first child's subtree)
 * so that a walk's node records share cache lines more often; topology,
 * child order and boxes are unchanged, so every walk visits the same nodes
 * in the same order and every result is bit-identical.  Run it after
 * fipt_scene_optimize and before the scene is given to a server.  The
 * radix-tree ranges of fipt_scene_debug_export no longer describe the tree
 * afterwards.  Not an operation of the paper. */
fipt_status fipt_scene_relayout(fipt_scene* scene, fipt_stream stream);

/* Replaces the radiance cache (cache [T,3] f32, original triangle order)
 * without rebuilding the BVH -- the refined-cache update between stages. */
fipt_status fipt_scene_set_cache(fipt_scene* scene, const float* cache, fipt_stream stream);
fipt_status fipt_scene_destroy(fipt_scene* scene);

/* Host-side scene facts: triangle count, ray-origin offset
 * eps = 1e-4 * largest extent (valid after the build has run; this call
 * synchronises the stream), and the workspace bytes in use. */
fipt_status fipt_scene_info(fipt_scene* scene, fipt_stream stream, int64_t* T, float* eps,
                            float* lo3, float* hi3);

/* Parity export of the LBVH (device outputs, any may be NULL):
 *  morton [T] u64 codes in sorted order; order [T] i32 triangle index at
 *  each sorted position; node_range [(T-1),3] i32 (first, last, split) of
 *  every internal node over sorted positions (FIPT_ERR_INVALID_ARG after
 *  fipt_scene_optimize); node_box [(T-1),6] f32 the node's box (lo xyz,
 *  hi xyz) = union of its two child boxes; node_child [(T-1),2] i32 the
 *  node's child references (>= 0 an internal node, < 0 the leaf ~ref). */
fipt_status fipt_scene_debug_export(fipt_scene* scene, uint64_t* morton, int32_t* order,
                                    int32_t* node_range, float* node_box, int32_t* node_child,
                                    fipt_stream stream);

/* ------------------------------------------------------------ rays */
/* Closest hit of nR rays o + t d, t > 0 (orig, dir [nR,3] f32; dir need
 * not be unit).  skip_tri [nR] i32 (nullable): a triangle each ray ignores.
 * Outputs [nR]: hit_tri i32 (original index, -1 = miss), hit_t f32 (+inf on
 * a miss), hit_front i32 (1 when d . ((v1-v0)x(v2-v0)) < 0).  Among equal t
 * the lower triangle index wins.  Watertight float32 test (Woop, Benthin,
 * Wald, JCGT 2013) with a float64 retry of exactly-zero edge functions. */
fipt_status fipt_trace_closest(fipt_scene* scene, const float* orig, const float* dir,
                               int64_t nR, const int32_t* skip_tri, int32_t* hit_tri,
                               float* hit_t, int32_t* hit_front, fipt_stream stream);

/* Pinhole first hits -> query records, one per pixel (P = nViews*W*H,
 * view-major, then row from the top, then column).
 *  cams [nViews,10] f32: eye xyz, forward xyz, up xyz, vertical fov (rad).
 *  right = normalize(fwd x up), up' = right x fwd; pixel (i, j) looks along
 *  normalize(fwd + sx right + sy up'), sx = (2(i+0.5)/W - 1) tan(fov/2) W/H,
 *  sy = (1 - 2(j+0.5)/H) tan(fov/2).
 *  out [P] fipt_query (16-byte aligned): x = eye + t d, n = unit face normal
 *  turned toward the camera, wo = -d, tri = hit; valid [P] i32 = 1 on a hit
 *  (records of misses are zero with tri = -1). */
fipt_status fipt_camera_queries(fipt_scene* scene, const float* cams, int32_t nViews, int32_t W,
                                int32_t H, fipt_query* out, int32_t* valid, fipt_stream stream);

/* Stream compaction of query records in order: the first max_out records
 * with valid != 0 are copied to out (16-byte aligned; may be NULL when
 * max_out is 0); pixel_of [max_out] i32 (nullable) receives their source
 * index; *n_out (device i64) the count written. */
fipt_status fipt_compact_workspace_size(int64_t P, size_t* bytes);
fipt_status fipt_compact_queries(const fipt_query* in, const int32_t* valid, int64_t P,
                                 int64_t max_out, fipt_query* out, int32_t* pixel_of,
                                 int64_t* n_out, void* workspace, size_t ws_bytes,
                                 fipt_stream stream);

/* ------------------------------------------------------------ bake */
/* Bakes the shading terms of Eq. 6 with the Fresnel split of Eq. 7 at N
 * query points (q [N] fipt_query, 8-byte aligned), by the Monte Carlo
 * estimator of Sec. 6 (stage 1, BRDF importance sampling) with the one-
 * segment cache query of Eq. 9: a ray leaves o = x + eps n, and its
 * incident radiance is L_e (front face only) + L' of the first triangle it
 * hits other than q.tri, or 0 on a miss.
 *  L_d: cosine-distributed directions; each sample contributes its radiance.
 *  L_s0/L_s1 at sigma_k: GGX half vectors drawn with density D(h)(n.h)
 *  (Walter et al. 2007), alpha = sigma_k^2, reflected to wi; a sample with
 *  n.wi <= 0 or wo.h <= 0 contributes 0; otherwise radiance times
 *  F0 w and F1 w, w = G (wo.h) / ((n.wo)(n.h)), G the separable Smith-GGX
 *  masking, F1 = (1 - wo.h)^5, F0 = 1 - F1.  Points with n.wo <= 1e-2
 *  get zero specular terms.
 * Outputs (f32): Ld [N,3], Ls0 [N,K,3], Ls1 [N,K,3]; each value is the sum
 * of its samples in sample order divided by the sample count, so results
 * are deterministic. */
fipt_status fipt_bake(fipt_scene* scene, const fipt_query* q, int64_t N,
                      const fipt_bake_params* params, float* Ld, float* Ls0, float* Ls1,
                      fipt_stream stream);

/* An order of the query points for fipt_bake (no counterpart in the paper):
 * order [N] DEVICE int32 receives the indices of the points sorted by the
 * 30-bit Morton code of their positions in the scene's bounding box
 * (stable: equal codes keep index order).  A warp bakes 32 consecutive
 * slots, and with this order its points lie close together, so their rays
 * start near each other and walk the tree alike (about 7 % faster on the
 * building floor than compacted pixel order; random order halves the
 * rate).  Workspace: fipt_query_order_workspace_size, 256-byte aligned. */
fipt_status fipt_query_order_workspace_size(int64_t N, size_t* bytes);
fipt_status fipt_query_order(fipt_scene* scene, const fipt_query* q, int64_t N, int32_t* order,
                             void* workspace, size_t ws_bytes, fipt_stream stream);

/* Environment radiance for rays that leave the scene (light through a
 * window, Sec. 8): env [H, W, 3] f32 device, caller-owned, kept alive while
 * set; NULL clears it (misses then bring 0).  Direction d maps to longitude
 * u = atan2(d.x, -d.z) / 2pi + 1/2 and colatitude v = acos(d.y) / pi;
 * texel (i, j) is centred at ((i + 1/2) / W, (j + 1/2) / H); lookups are
 * bilinear, wrapping in u and clamped in v.  Used by fipt_bake,
 * fipt_bake_refine and the server's batched bakes. */
fipt_status fipt_scene_set_environment(fipt_scene* scene, const float* env, int32_t W, int32_t H);

/* Voxel radiance cache (Sec. 4.2): L' as an R^3 grid spanned over the
 * scene box, average-pooled from input pixels at their first hits and
 * queried at the voxel containing a hit point (the paper uses R = 256).
 * fipt_voxel_cache_build pools P pixels: point p at x[p * x_stride + 0..2]
 * (x_stride 3 for a plain [P,3] array, 10 to read fipt_query records) with
 * radiance L [P,3] f32; pixels are assigned to cell
 * floor((x - lo) * (R / (hi - lo))) per axis (clamped to [0, R-1]), each
 * operation one IEEE double rounding; grid [R,R,R,4] f32 (index [z][y][x],
 * 16-byte aligned, caller-owned) receives (mean rgb, pixel count), zero for
 * empty voxels; each mean is summed in pixel order in FP64.  R in
 * [1, 1024]; workspace from fipt_voxel_cache_workspace_size(P). */
fipt_status fipt_voxel_cache_workspace_size(int64_t P, size_t* bytes);
fipt_status fipt_voxel_cache_build(fipt_scene* scene, const float* x, int64_t x_stride,
                                   const float* L, int64_t P, int32_t R, float* grid,
                                   void* workspace, size_t ws_bytes, fipt_stream stream);
/* Uses a built grid (kept alive by the caller) as the cache L' of the bake,
 * the refinement and the server's batches instead of the per-triangle
 * values; NULL returns to per-triangle values. */
fipt_status fipt_scene_set_voxel_cache(fipt_scene* scene, const float* grid, int32_t R);

/* ------------------------------------------------ emitter extraction */
/* Emitter extraction (Sec. 4.4, Eq. 12).  Step 1: n_per_tri locations
 * uniform on every triangle, for the caller to evaluate its emission-mask
 * field alpha at: point j of triangle t uses the Philox words of counter
 * (t, j, 0x400, request_id), key (seed lo, seed hi); u1, u2 from the first
 * two words (top 24 bits times 2^-24), barycentrics (1 - sqrt(u1),
 * sqrt(u1) (1 - u2), sqrt(u1) u2) on the triangle's float vertices in f32.
 * x: device f32 [T * n_per_tri, 3] (triangle-major, original triangle
 * order, caller-owned).  n_per_tri in [1, 2^20] (the paper uses 100), T *
 * n_per_tri < 2^39. */
fipt_status fipt_emitter_sample_points(fipt_scene* scene, uint64_t seed, uint32_t request_id,
                                       int32_t n_per_tri, float* x, fipt_stream stream);
/* Step 2: triangle t is an emitter when the mean of
 * alpha[t * n_per_tri .. +n_per_tri) (device f32, summed in order in FP64,
 * divided by n_per_tri) is > threshold (0.01 in the paper, compared in
 * FP64).  is_emitter: device u8 [T] (0/1); mean_alpha: device f64 [T] or
 * NULL. */
fipt_status fipt_emitter_classify(const float* alpha, int64_t T, int32_t n_per_tri, float threshold,
                                  double* mean_alpha, uint8_t* is_emitter, fipt_stream stream);
/* Step 3: with zero reflectance at emitters the L1 fit of Eq. 12 has the
 * closed form L_e = per-channel median of the radiance of the input pixels
 * whose first hit is the triangle.  tri: device i32, pixel p's triangle at
 * tri[p * tri_stride] (stride 10 reads the id of fipt_query records; < 0 or
 * >= T: no triangle); rgb: device f32 [P,3]; is_emitter: device u8 [T].
 * Le: device f32 [T,3] receives the lower median (sorted value at index
 * (c - 1) / 2 of the c pixels) of emitter triangles, 0 for other triangles
 * and for emitters no pixel hits; count: device i32 [T] or NULL, the pixels
 * per emitter triangle.  Values order as IEEE totalOrder (NaN above +inf).
 * Workspace from fipt_emitter_radiance_workspace_size(P, T). */
fipt_status fipt_emitter_radiance_workspace_size(int64_t P, int64_t T, size_t* bytes);
fipt_status fipt_emitter_radiance(const int32_t* tri, int64_t tri_stride, const float* rgb, int64_t P,
                                  const uint8_t* is_emitter, int64_t T, float* Le, int32_t* count,
                                  void* workspace, size_t ws_bytes, fipt_stream stream);
/* Replaces the scene's emission L_e (device f32 [T,3], original order) and
 * rebuilds the emitter table the refinement samples, without rebuilding
 * the BVH. */
fipt_status fipt_scene_set_emission(fipt_scene* scene, const float* Le, fipt_stream stream);

/* Per-triangle materials for the refinement (stage-2 estimates in the
 * paper): albedo [T,3], roughness [T], metallic [T] f32, original order. */
fipt_status fipt_scene_set_materials(fipt_scene* scene, const float* albedo, const float* rough,
                                     const float* metal, fipt_stream stream);

/* Stage-3 path-traced refinement of the shading terms (Sec. 4.3, Eq. 10,
 * with multiple importance sampling as Sec. 6 states).  A sample starts as
 * in fipt_bake (same lobe, same Philox stream) and grows its path through
 * surfaces whose roughness is <= sigma_c (0.6 in the paper), sampling the
 * full BRDF of Eq. 1 there (diffuse lobe with probability
 * clamp(mean(k_d)/(mean(k_d)+mean(k_s)), 0.1, 0.9)), until it reaches an
 * emitter (L_e, front face) or a rougher surface (the cache L'); at most
 * max_depth vertices beyond the first hit.  mis != 0: every vertex also
 * samples a point on the emitters (area-uniform over all triangles with
 * L_e > 0) and the two strategies are combined by the power heuristic.
 * Philox counters: lobe direction at x (pid, s, lobe, rid); emitter sample
 * at x (pid, s, lobe|0x100, rid); BRDF at vertex i (pid, s, lobe|i<<9, rid);
 * emitter sample at vertex i (pid, s, lobe|i<<9|0x100, rid).
 * Outputs as fipt_bake: each value is the mean of its samples' values,
 * summed in sample order.  per_sample (nullable, device f32
 * [N, 1+K, max(spp), 6]) receives every sample's value (L_d uses the first
 * 3 values, L_s0 / L_s1 the two triples; zeros past a lobe's sample
 * count).  params->stats (NULL, or 4 device u64 counters) receives, added,
 * the rays traced (path segments and shadow rays), nodes visited and
 * triangles tested, and the deepest stack (max).  Requires
 * fipt_scene_set_materials.
 * workspace: device, 256-byte aligned, at least the bytes
 * fipt_bake_refine_workspace_size gives for the same N, params and
 * max_depth (the path state of up to 16,777,216 samples at a time, 184
 * bytes each, about 3.1 GB; larger calls run in chunks of whole points);
 * owned by the caller, in use until the stream reaches the end of the call.
 * spp_diffuse + K * spp_specular above 16,777,216 is FIPT_ERR_INVALID_ARG;
 * a workspace below the size is FIPT_ERR_WORKSPACE.  max_depth > 15 makes
 * the call wait for the stream every 16 path depths to stop once every
 * path has ended. */
fipt_status fipt_bake_refine_workspace_size(int64_t N, const fipt_bake_params* params,
                                            int32_t max_depth, size_t* bytes);
fipt_status fipt_bake_refine(fipt_scene* scene, const fipt_query* q, int64_t N,
                             const fipt_bake_params* params, float sigma_c, int32_t max_depth,
                             int32_t mis, float* Ld, float* Ls0, float* Ls1, float* per_sample,
                             void* workspace, size_t ws_bytes, fipt_stream stream);

/* ------------------------------------------------------------ render */
/* Factorized render, Eq. 5 with k_d = a(1-m), k_s = 0.04(1-m) + a m (Eq. 1)
 * and the roughness lerp of Eq. 8: sigma is clamped to
 * [sigma_grid[0], sigma_grid[K-1]], segment i is the largest i <= K-2 with
 * sigma_grid[i] <= sigma.  Inputs: tables as produced by fipt_bake;
 * sigma_grid [K] HOST f32 increasing, K in [2, 8] (a lerp needs two
 * nodes; other K is FIPT_ERR_INVALID_ARG); albedo [N,3], rough [N], metal [N]
 * f32.  Outputs: Lr [N,3] f32.  When Lgt [N,3] is given, *loss (device
 * f64) = sum over points with mask != 0 (mask [N] u8, NULL = all) and
 * channels of (Gamma(Lr) - Gamma(Lgt))^2 (Eq. 14 with alpha = 0),
 * Gamma(x) = sRGB(log(1 + max(x, 0))); summed in a fixed order. */
fipt_status fipt_render_workspace_size(int64_t N, size_t* bytes);
fipt_status fipt_render_fwd(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                            int32_t K, const float* sigma_grid, const float* albedo,
                            const float* rough, const float* metal, const float* Lgt,
                            const uint8_t* mask, float* Lr, double* loss, void* workspace,
                            size_t ws_bytes, fipt_stream stream);

/* fipt_render_fwd without a workspace, for callers that cannot allocate
 * device memory when they render (their device memory is a fixed pool
 * sized at start-up, or they run on threads that must not take an
 * allocator's lock).  The paper has no counterpart; this is a library convenience.
 * Same arguments and results as fipt_render_fwd; the loss partial sums live
 * in a 1 MiB array compiled into the library, present on every GPU that
 * loads it until the process exits.  N may be at most
 * FIPT_NOALLOC_RENDER_MAX_BLOCKS * 128 = 16,777,216 points; larger N returns
 * FIPT_ERR_INVALID_ARG without launching.  Allocates nothing: the first call
 * on a device looks up the array's device address (cudaGetSymbolAddress,
 * with that device current) and keeps it; later calls check with
 * cudaPointerGetAttributes that the driver still knows that address as
 * memory of the device, and look it up again if not (after a
 * cudaDeviceReset, say).  Make the first call on each device before any
 * stream capture.  Every call on a device shares the one array: calls that overlap
 * on the GPU (different streams, no ordering between them) race and may
 * return a wrong loss; serialise them on one stream.  Each call overwrites
 * every partial it reads, so no clearing is needed between calls. */
#define FIPT_NOALLOC_RENDER_MAX_BLOCKS 131072
fipt_status fipt_render_fwd_noalloc(const float* Ld, const float* Ls0, const float* Ls1,
                                    int64_t N, int32_t K, const float* sigma_grid,
                                    const float* albedo, const float* rough, const float* metal,
                                    const float* Lgt, const uint8_t* mask, float* Lr,
                                    double* loss, fipt_stream stream);

/* Gradient of that loss times *grad_loss (device f64 scalar, NULL = 1)
 * with respect to albedo [N,3], rough [N], metal [N] (f32 outputs).  The
 * derivative in sigma is 0 where sigma is outside the grid; at grid nodes
 * it is the right segment's slope. */
fipt_status fipt_render_bwd(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                            int32_t K, const float* sigma_grid, const float* albedo,
                            const float* rough, const float* metal, const float* Lgt,
                            const uint8_t* mask, const double* grad_loss, float* g_albedo,
                            float* g_rough, float* g_metal, fipt_stream stream);

/* Forward, loss and gradient in one pass (one training step's render):
 * writes Lr and *loss as fipt_render_fwd with the same Lgt and mask, and
 * g_albedo [N,3], g_rough [N], g_metal [N] as fipt_render_bwd with
 * grad_loss = NULL (an upstream gradient of 1), reading each input once
 * instead of twice.  Lgt, loss, Lr and the gradient outputs are required;
 * workspace as fipt_render_fwd (fipt_render_workspace_size bytes, 8-byte
 * aligned, caller-owned).  Sec. 4.1, Eq. 5, 8, 14. */
fipt_status fipt_render_fwd_grad(const float* Ld, const float* Ls0, const float* Ls1, int64_t N,
                                 int32_t K, const float* sigma_grid, const float* albedo,
                                 const float* rough, const float* metal, const float* Lgt,
                                 const uint8_t* mask, float* Lr, double* loss, float* g_albedo,
                                 float* g_rough, float* g_metal, void* workspace, size_t ws_bytes,
                                 fipt_stream stream);

/* Multiplies the gradients of fipt_render_fwd_grad in place by the
 * upstream gradient *grad_loss (device f64 scalar, read on the device and
 * rounded to f32 as fipt_render_bwd does); a factor of exactly 1 leaves
 * them unchanged without touching them. */
fipt_status fipt_render_grad_scale(int64_t N, const double* grad_loss, float* g_albedo,
                                   float* g_rough, float* g_metal, fipt_stream stream);

/* ------------------------------------------------------------ emitters */
/* Per-triangle rendering error (Sec. 4.4: rendering without emission
 * leaves large error on emitters).  tri: first-hit triangle of each pixel
 * (-1 = none, ignored), pixel p's index at tri[p * tri_stride] (i32; 1 for
 * a plain array, 10 to read the tri field of fipt_query records); Lr, Lgt
 * [P,3] f32.  Outputs: err_sum [T] f64
 * = sum of ||Lr - Lgt||^2 over the triangle's pixels, summed in pixel
 * order; count [T] i32.  Pixels are grouped by a stable radix sort on the
 * triangle index held in the workspace. */
fipt_status fipt_tri_error_workspace_size(int64_t P, int64_t T, size_t* bytes);
fipt_status fipt_tri_error(const int32_t* tri, int64_t tri_stride, const float* Lr,
                           const float* Lgt, int64_t P, int64_t T, double* err_sum, int32_t* count, void* workspace,
                           size_t ws_bytes, fipt_stream stream);

/* ------------------------------------------------------------ serving */
/* A request loop over resident scenes with continuous batching (a serving
 * pattern around the bake; the paper runs one bake per scene offline).
 *
 * fipt_server_create allocates one device arena of hbm_budget bytes (the
 * admission budget), two work queues (device descriptors plus a
 * host-mapped control block and per-chunk done flags), and starts a host
 * scheduler thread.  Requests are admitted in arrival order as arena space
 * frees up.  Requests run in two device-resident loops, kernels whose
 * warps stay resident on every SM and take warp items as the scheduler
 * publishes them, without a launch per request:
 *  - the bake loop (all block slots of 64 threads but two per SM): warp
 *    items of 32 points of one chunk and one lobe, one atomic add each.
 *    The scheduler keeps bake items published ahead of the loop and not
 *    yet taken -- two per resident warp, and at least max_batch_rays rays
 *    -- in chunks of up to chunk_points points: the oldest request first,
 *    up to a quarter of that, then the requests with the least remaining
 *    work -- so a request that arrives while others run joins their warps
 *    on the device;
 *  - the render loop (two block slots per SM): a render request
 *    (Eq. 5, 8, 14 and the loss gradient for an upstream gradient of 1)
 *    is published whole, in items of 512 rows, and starts as soon as its
 *    inputs are on the device, whatever the bake loop holds.
 * The scheduler stops the loops after a millisecond without work and
 * starts them again when new work is published.  Scene environment maps
 * and voxel caches must be set before a scene is added.
 * A bake chunk keeps the request-local Philox counters (point_base = its
 * offset in the request) and a render item sums the loss in the render
 * kernels' order, so every result is bit-identical to a standalone
 * fipt_bake / fipt_render_fwd_grad of the same request (where a chunk's
 * warps group points differently from the standalone bake, with the
 * float32 caveat stated at fipt_bake_params.order).
 * All host buffers of a request must stay valid until it completes; pinned
 * (page-locked) buffers let copies overlap compute.  Every wait is bounded:
 * the scheduler polls events and the mapped flags; a bake warp that has
 * polled the published count about half a second in vain ends the launch
 * (its item, like every item a stopped launch holds, runs first in the
 * next launch), and a render warp that has found no render work for as
 * long ends the render launch. */
#define FIPT_REQ_BAKE 0
#define FIPT_REQ_RENDER 1

typedef struct fipt_server fipt_server;

typedef struct fipt_request {
    int32_t kind;                 /* FIPT_REQ_BAKE or FIPT_REQ_RENDER */
    int32_t target;               /* scene id (bake) or table id (render) */
    int64_t n;                    /* points (bake) or table rows (render) */
    int64_t first;                /* render: first table row */
    /* bake: HOST queries [n]; params (point_base ignored, stats must be
     * NULL); HOST outputs Ld [n,3], Ls0 [n,K,3], Ls1 [n,K,3] */
    const fipt_query* queries;
    fipt_bake_params params;
    float* Ld;
    float* Ls0;
    float* Ls1;
    /* render (Eq. 5, 8, 14 over table rows [first, first+n)): HOST inputs
     * albedo [n,3], rough [n], metal [n], Lgt [n,3]; HOST outputs (each may
     * be NULL) Lr [n,3], loss [1], g_albedo [n,3], g_rough [n], g_metal [n] */
    const float* albedo;
    const float* rough;
    const float* metal;
    const float* Lgt;
    float* Lr;
    double* loss;
    float* g_albedo;
    float* g_rough;
    float* g_metal;
} fipt_request;

typedef struct fipt_server_stats {
    uint64_t batches;                /* launches of the resident bake loop */
    uint64_t chunks;                 /* bake chunks published */
    uint64_t rays;                   /* bake rays completed */
    uint64_t max_requests_per_batch; /* most bake requests with chunks on the device at once */
    uint64_t bytes_in_use;           /* arena bytes held by admitted requests */
    uint64_t peak_bytes;
    uint64_t pending;                /* requests waiting for admission */
} fipt_server_stats;

fipt_status fipt_server_create(fipt_ctx* ctx, size_t hbm_budget, int64_t max_batch_rays,
                               int64_t chunk_points, fipt_server** out);
/* Registers a built scene (kept alive by the caller) -> *id for bake requests. */
fipt_status fipt_server_add_scene(fipt_server* srv, fipt_scene* scene, int32_t* id);
/* Registers resident device tables (Ld [N,3], Ls0/Ls1 [N,K,3]; sigma_grid
 * HOST [K]) -> *id for render requests.  Kept alive by the caller. */
fipt_status fipt_server_add_table(fipt_server* srv, const float* Ld, const float* Ls0,
                                  const float* Ls1, int64_t N, int32_t K,
                                  const float* sigma_grid, int32_t* id);
/* Queues a request (the struct is copied) -> *ticket.  A request needing
 * more device memory than the whole budget completes at once with result
 * FIPT_ERR_BUDGET; bad ids / parameters return FIPT_ERR_INVALID_ARG. */
fipt_status fipt_server_submit(fipt_server* srv, const fipt_request* req, uint64_t* ticket);
/* *done = 1 once the request's outputs are in its host buffers; *result is
 * its status (FIPT_OK, FIPT_ERR_BUDGET, FIPT_ERR_DEVICE_CHECK, ...). */
fipt_status fipt_server_poll(fipt_server* srv, uint64_t ticket, int32_t* done, fipt_status* result);
/* Blocks until done or timeout_us elapses (then returns FIPT_ERR_TIMEOUT). */
fipt_status fipt_server_wait(fipt_server* srv, uint64_t ticket, int64_t timeout_us,
                             fipt_status* result);
/* Host steady-clock seconds at submit, admission and completion. */
fipt_status fipt_server_times(fipt_server* srv, uint64_t ticket, double* t_submit, double* t_admit,
                              double* t_done);
/* Forgets a finished request. */
fipt_status fipt_server_release(fipt_server* srv, uint64_t ticket);
fipt_status fipt_server_get_stats(fipt_server* srv, fipt_server_stats* out);
/* Failure handling.  When a submission to the device fails (a descriptor
 * copy, a start of a loop) or device work fails, the
 * server tells the loops to stop, starts no new work, and every unfinished
 * request ends with that error (its *result) -- each one only after none
 * of its input copy, kernels or output copies is still queued, so a caller
 * whose wait returns may free or reuse the request's host buffers at once.
 * Requests already copying their outputs keep their own results.
 * Test hook (the paper has no counterpart): after the next after_launches
 * device submissions (a publication of bake or render descriptors, a start
 * of either loop) the following one fails with FIPT_ERR_CUDA on the host
 * instead of reaching the device. */
fipt_status fipt_server_inject_launch_failure(fipt_server* srv, int64_t after_launches);
/* Test hook (host only): a request's input copies (at admission) and its
 * output copies (at completion) each count as one copy step; after
 * `after_steps` more steps, the next one is treated as refused, as if one
 * of its cudaMemcpyAsync calls had returned an error.  A request whose copy
 * step is refused -- injected or real -- ends with FIPT_ERR_CUDA once what
 * it did enqueue has completed, without running if its inputs were
 * refused; other requests and the server go on. */
fipt_status fipt_server_inject_copy_failure(fipt_server* srv, int64_t after_steps);
/* Cancels requests not yet admitted (result FIPT_ERR_NOT_FOUND), drains
 * admitted work, joins the scheduler and frees the arena. */
fipt_status fipt_server_destroy(fipt_server* srv);

/* First-fit arena bookkeeping the server uses for admission (host only,
 * offsets in [0, bytes), 256-byte granularity, neighbours coalesce). */
typedef struct fipt_arena fipt_arena;
fipt_status fipt_arena_create(size_t bytes, fipt_arena** out);
fipt_status fipt_arena_alloc(fipt_arena* a, size_t bytes, size_t* offset);  /* FIPT_ERR_BUDGET when full */
fipt_status fipt_arena_free(fipt_arena* a, size_t offset, size_t bytes);
fipt_status fipt_arena_info(fipt_arena* a, size_t* used, size_t* peak, size_t* largest_free);
fipt_status fipt_arena_destroy(fipt_arena* a);

/* ------------------------------------------------------------ checks */
/* Philox4x32-10 on the device (parity check of the sampler's stream):
 * ctr [n,4] u32, key [n,2] u32 -> out [n,4] u32. */
fipt_status fipt_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n,
                              uint32_t* out, fipt_stream stream);
/* The emitter sampler's split of a sample index i into (triangle i / n,
 * sample i mod n) divides by the invariant n with one multiply-high
 * (Granlund and Montgomery 1994); the paper has no counterpart.  out[k] =
 * i[k] / n by that same routine, on the host (on_device = 0: i and out
 * HOST arrays, stream ignored) or in a kernel (on_device != 0: DEVICE
 * arrays on the stream).  n >= 1. */
fipt_status fipt_debug_divide(uint32_t n, const uint32_t* i, int64_t count, uint32_t* out,
                              int32_t on_device, fipt_stream stream);
/* The server's resident loop on a queue that nothing ever publishes to
 * (check of its bounded wait; no counterpart in the paper): one block per
 * SM, every warp takes one item and waits for it; after wait_polls naps
 * (each at most about 32 microseconds) a warp gives up and the whole
 * launch leaves.  Blocks the calling thread until the kernel has ended by
 * itself.  -> *quit = the launch's quit flag (1), *orphans = items the
 * warps left behind (one per warp), *warps = warps launched, *seconds =
 * the kernel's duration.  1 <= wait_polls <= 65536. */
fipt_status fipt_debug_serve_wait_bound(int32_t wait_polls, int32_t* quit, int32_t* orphans,
                                        int32_t* warps, double* seconds);
/* The order the server gives a bake's points (the order of
 * fipt_query_order, computed on the host by a threaded radix sort): q [n]
 * HOST, lo [3] / hi [3] HOST box -> order [n] HOST.  Check entry point; no
 * counterpart in the paper. */
fipt_status fipt_debug_host_query_order(const fipt_query* q, int64_t n, const float* lo, const float* hi,
                                        int32_t* order);

#ifdef __cplusplus
}
#endif
#endif /* FIPT_H */
