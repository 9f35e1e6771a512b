/*
 * FP64 CPU oracle for the factorized shading-term bake of
 * "Factorized Inverse Path Tracing" (Wu et al., ICCV 2023, arXiv 2304.05669).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path, and the
 * CUDA path never calls it.
 *
 * Everything here is the plain definition, written for a reader who checks
 * it against the paper by eye:
 *   - Philox4x32-10 counter-based RNG (Salmon et al., SC'11).
 *   - Shading integrals of Eq. 6 with the Fresnel split of Eq. 7, estimated
 *     by BRDF importance sampling (Sec. 6, stage 1) with the one-segment
 *     cache query of Eq. 9: L_i = front-face L_e + L'(x1) at the first hit.
 *   - Closest hit by brute force or by an independent top-down
 *     spatial-median BVH; FP64 Moeller-Trumbore with inclusive edges.
 *   - Morton codes and the binary radix tree over them (the bit-exact
 *     targets for the device LBVH), built top-down by splitting each key
 *     range at its highest differing bit.
 *
 * Compile with -ffp-contract=off: the Morton quantisation must be a chain
 * of individually rounded IEEE double operations.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OPI 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11).  Ten rounds; the key is bumped by the   */
/* Weyl constants between rounds.                                       */
/* ------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u, PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u, PHILOX_W1 = 0xBB67AE85u;

static void philox10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) philox10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* A 32-bit output word -> uniform in [0,1): its top 24 bits times 2^-24. */
static double u24(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

/* Jittered stratification of the lobe samples at a query point (the
 * paper fixes no sampler; this is the reading of its importance-sampled
 * estimates used here).  The S samples of a (point, lobe) pair cover an
 * nx x ny grid over (u1, u2), nx the largest divisor of S with nx^2 <= S
 * and ny = S / nx: sample s lies in cell (s mod nx, s div nx), placed in
 * it by the pair's own Philox uniforms.  Every cell holds one sample, each
 * sample is uniform over [0,1)^2 and the pairs stay independent, so each
 * estimate keeps its expectation and its variance does not grow. */
static int strat_cols(int S)
{
    int nx = 1;
    for (int d = 1; (int64_t)d * d <= S; ++d)
        if (S % d == 0) nx = d;
    return nx;
}

/* The stratified uniform is formed in float32, fl(fl(cell + r) / n) capped
 * at the largest float below 1, exactly as the kernels form it, so the
 * uniforms stay bit-identical on both sides (r, a 24-bit uniform, is exact
 * in float32; a sample at the far edge of its cell can round onto the next
 * cell's boundary, about 2^-22 of them, a float32 quantisation like the
 * 24-bit uniform's own). */
static double strat_one(uint32_t cell, int n, double r)
{
    const float u = ((float)cell + (float)r) / (float)n;
    return (double)fminf(u, 0x1.fffffep-1f);
}

static void strat_uv(uint32_t s, int S, double* u1, double* u2)
{
    if (S <= 0) return;
    const int nx = strat_cols(S), ny = S / nx;
    const uint32_t i = s % (uint32_t)nx, j = s / (uint32_t)nx;
    *u1 = strat_one(i, nx, *u1);
    *u2 = strat_one(j, ny, *u2);
}

/* strat_uv over arrays (pins of the stratification). */
void oracle_strat_uv(int S, const uint32_t* s, const double* r1, const double* r2, int64_t n, double* u1,
                     double* u2)
{
    for (int64_t k = 0; k < n; ++k) {
        u1[k] = r1[k];
        u2[k] = r2[k];
        strat_uv(s[k], S, &u1[k], &u2[k]);
    }
}

/* ------------------------------------------------------------------ */
/* Small vector helpers                                                 */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }
static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1]*b[2] - a[2]*b[1];
    r[1] = a[2]*b[0] - a[0]*b[2];
    r[2] = a[0]*b[1] - a[1]*b[0];
}
static void sub3(const double a[3], const double b[3], double r[3]) { r[0]=a[0]-b[0]; r[1]=a[1]-b[1]; r[2]=a[2]-b[2]; }
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }
static void normalize3(double a[3]) { double l = norm3(a); a[0] /= l; a[1] /= l; a[2] /= l; }

/* ------------------------------------------------------------------ */
/* Scene                                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    double v0[3], v1[3], v2[3];
    double e1[3], e2[3];
    double ng[3];        /* (v1-v0) x (v2-v0), not normalised */
    double area2;        /* |ng| = twice the area */
    double h[3];         /* altitude onto the edge opposite vertex i */
    double lo[3], hi[3]; /* bounding box */
    double c[3];         /* box centre, used to split the BVH */
} otri;

typedef struct {
    double lo[3], hi[3];
    int left, right;     /* children, or -1 for a leaf */
    int start, count;    /* triangle range in idx[] for a leaf */
} onode;

typedef struct {
    int64_t T;
    otri* tri;
    double* Le;          /* T x 3 */
    double* cache;       /* T x 3 */
    onode* node;
    int nnode;
    int* idx;
    double slo[3], shi[3]; /* scene box from float vertex min / max */
    double L;              /* largest extent of the scene box */
    double diag;           /* length of its diagonal */
    double eps;            /* ray-origin offset, 1e-4 * L */
    double* env;           /* environment radiance [H][W][3] (NULL: misses bring 0) */
    int env_w, env_h;
    double* vox;           /* voxel radiance cache [R^3][4]: mean rgb, pixel count (NULL: per-triangle) */
    int vox_r;
} oscene;

static int build_node(oscene* S, int start, int count, int* cap)
{
    if (S->nnode >= *cap) {
        *cap *= 2;
        S->node = (onode*)realloc(S->node, sizeof(onode) * (size_t)(*cap));
    }
    int id = S->nnode++;
    onode nd;
    for (int a = 0; a < 3; ++a) { nd.lo[a] = INFINITY; nd.hi[a] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = start; i < start + count; ++i) {
        const otri* t = &S->tri[S->idx[i]];
        for (int a = 0; a < 3; ++a) {
            if (t->lo[a] < nd.lo[a]) nd.lo[a] = t->lo[a];
            if (t->hi[a] > nd.hi[a]) nd.hi[a] = t->hi[a];
            if (t->c[a] < clo[a]) clo[a] = t->c[a];
            if (t->c[a] > chi[a]) chi[a] = t->c[a];
        }
    }
    nd.left = nd.right = -1;
    nd.start = start;
    nd.count = count;
    if (count > 4) {
        int ax = 0;
        for (int a = 1; a < 3; ++a) if (chi[a] - clo[a] > chi[ax] - clo[ax]) ax = a;
        double mid = 0.5 * (clo[ax] + chi[ax]);
        int i = start, j = start + count - 1;
        while (i <= j) {                       /* partition about the midpoint */
            if (S->tri[S->idx[i]].c[ax] < mid) ++i;
            else { int tmp = S->idx[i]; S->idx[i] = S->idx[j]; S->idx[j] = tmp; --j; }
        }
        int nl = i - start;
        if (nl == 0 || nl == count) nl = count / 2;   /* all centres equal: halve */
        S->node[id] = nd;
        int l = build_node(S, start, nl, cap);
        int r = build_node(S, start + nl, count - nl, cap);
        S->node[id].left = l;
        S->node[id].right = r;
        S->node[id].count = 0;
        return id;
    }
    S->node[id] = nd;
    return id;
}

oscene* oracle_scene_create(const float* V, int64_t nV, const int32_t* F, int64_t T,
                            const float* Le, const float* cache)
{
    oscene* S = (oscene*)calloc(1, sizeof(oscene));
    S->T = T;
    S->tri = (otri*)calloc((size_t)(T > 0 ? T : 1), sizeof(otri));
    S->Le = (double*)calloc((size_t)(3 * (T > 0 ? T : 1)), sizeof(double));
    S->cache = (double*)calloc((size_t)(3 * (T > 0 ? T : 1)), sizeof(double));
    float flo[3] = {INFINITY, INFINITY, INFINITY}, fhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nV; ++i)
        for (int a = 0; a < 3; ++a) {
            if (V[3*i+a] < flo[a]) flo[a] = V[3*i+a];
            if (V[3*i+a] > fhi[a]) fhi[a] = V[3*i+a];
        }
    S->L = 0.0;
    for (int a = 0; a < 3; ++a) {
        S->slo[a] = nV ? flo[a] : 0.0;
        S->shi[a] = nV ? fhi[a] : 0.0;
        if (S->shi[a] - S->slo[a] > S->L) S->L = S->shi[a] - S->slo[a];
    }
    double dg[3]; sub3(S->shi, S->slo, dg);
    S->diag = norm3(dg);
    S->eps = 1e-4 * S->L;
    for (int64_t t = 0; t < T; ++t) {
        otri* r = &S->tri[t];
        for (int a = 0; a < 3; ++a) {
            r->v0[a] = V[3*F[3*t+0]+a];
            r->v1[a] = V[3*F[3*t+1]+a];
            r->v2[a] = V[3*F[3*t+2]+a];
        }
        sub3(r->v1, r->v0, r->e1);
        sub3(r->v2, r->v0, r->e2);
        cross3(r->e1, r->e2, r->ng);
        r->area2 = norm3(r->ng);
        double e12[3]; sub3(r->v2, r->v1, e12);
        double l0 = norm3(e12), l1 = norm3(r->e2), l2 = norm3(r->e1);
        r->h[0] = l0 > 0 ? r->area2 / l0 : 0.0;
        r->h[1] = l1 > 0 ? r->area2 / l1 : 0.0;
        r->h[2] = l2 > 0 ? r->area2 / l2 : 0.0;
        for (int a = 0; a < 3; ++a) {
            r->lo[a] = fmin(r->v0[a], fmin(r->v1[a], r->v2[a]));
            r->hi[a] = fmax(r->v0[a], fmax(r->v1[a], r->v2[a]));
            r->c[a] = 0.5 * (r->lo[a] + r->hi[a]);
        }
        for (int a = 0; a < 3; ++a) {
            S->Le[3*t+a] = Le ? Le[3*t+a] : 0.0;
            S->cache[3*t+a] = cache ? cache[3*t+a] : 0.0;
        }
    }
    S->idx = (int*)malloc(sizeof(int) * (size_t)(T > 0 ? T : 1));
    for (int64_t t = 0; t < T; ++t) S->idx[t] = (int)t;
    int cap = 1024;
    S->node = (onode*)malloc(sizeof(onode) * (size_t)cap);
    S->nnode = 0;
    if (T > 0) build_node(S, 0, (int)T, &cap);
    return S;
}

void oracle_scene_destroy(oscene* S)
{
    if (!S) return;
    free(S->tri); free(S->Le); free(S->cache); free(S->node); free(S->idx); free(S->env); free(S->vox);
    free(S);
}

/* Voxel of a point: grid of R cells per axis over the scene box [lo, hi]
 * (from the float vertices), cell = floor((p - lo) * (R / (hi - lo))) clamped
 * to [0, R-1], each operation one IEEE double rounding (as the Morton
 * quantisation).  frac (nullable) receives the position inside the cell. */
static int64_t voxel_of(const oscene* S, int R, const double p[3], double frac[3])
{
    int64_t idx[3];
    for (int a = 0; a < 3; ++a) {
        double ext = S->shi[a] - S->slo[a];
        double f = ext > 0 ? (p[a] - S->slo[a]) * ((double)R / ext) : 0.0;
        double fl = floor(f);
        if (frac) frac[a] = f - fl;
        if (fl < 0) { fl = 0; if (frac) frac[a] = 0.5; }
        if (fl > R - 1) { fl = R - 1; if (frac) frac[a] = 0.5; }
        idx[a] = (int64_t)fl;
    }
    return (idx[2] * R + idx[1]) * R + idx[0];
}

/* Average pooling of pixel radiance onto the voxel grid (Sec. 4.2): every
 * pixel p with first-hit point x[p] adds its radiance L[p] to its voxel;
 * out[v] = (mean rgb, count), zero where no pixel fell. */
void oracle_voxel_pool(const oscene* S, const float* x, const float* L, int64_t P, int R, double* out)
{
    const int64_t nv = (int64_t)R * R * R;
    for (int64_t v = 0; v < 4 * nv; ++v) out[v] = 0.0;
    for (int64_t p = 0; p < P; ++p) {
        double q[3] = {x[3*p], x[3*p+1], x[3*p+2]};
        int64_t v = voxel_of(S, R, q, NULL);
        for (int c = 0; c < 3; ++c) out[4*v+c] += L[3*p+c];
        out[4*v+3] += 1.0;
    }
    for (int64_t v = 0; v < nv; ++v)
        if (out[4*v+3] > 0) for (int c = 0; c < 3; ++c) out[4*v+c] /= out[4*v+3];
}

/* Uses a pooled grid (as oracle_voxel_pool writes it) as the cache L'
 * looked up at the voxel containing a hit; NULL returns to per-triangle. */
void oracle_scene_set_voxel_cache(oscene* S, const double* grid, int R)
{
    free(S->vox);
    S->vox = NULL;
    S->vox_r = 0;
    if (!grid || R <= 0) return;
    size_t n = 4 * (size_t)R * R * R;
    S->vox = (double*)malloc(sizeof(double) * n);
    memcpy(S->vox, grid, sizeof(double) * n);
    S->vox_r = R;
}

/* Cache radiance at a hit point: the voxel grid when set, else the hit
 * triangle's value. */
static void cache_at(const oscene* S, int32_t id, const double p[3], double C[3])
{
    if (S->vox) {
        int64_t v = voxel_of(S, S->vox_r, p, NULL);
        for (int c = 0; c < 3; ++c) C[c] = S->vox[4*v+c];
    } else {
        for (int c = 0; c < 3; ++c) C[c] = S->cache[3*id+c];
    }
}

/* Whether a float32 hit point may fall in a neighbouring voxel: some
 * coordinate lies within 1e-3 of a cell face (a float32 hit point is off
 * by ~1e-6 of the scene size, ~1e-4 of a 256-cell voxel) and the cell
 * across that face is inside the grid (beyond the grid, both sides clamp
 * into the same border cell). */
static int voxel_ambiguous(const oscene* S, const double p[3])
{
    if (!S->vox) return 0;
    const int R = S->vox_r;
    double fr[3];
    int64_t v = voxel_of(S, R, p, fr);
    int64_t ix[3] = {v % R, (v / R) % R, v / ((int64_t)R * R)};
    for (int a = 0; a < 3; ++a) {
        if (fr[a] < 1e-3 && ix[a] > 0) return 1;
        if (fr[a] > 1.0 - 1e-3 && ix[a] < R - 1) return 1;
    }
    return 0;
}

/* Environment radiance seen by rays that leave the scene (a window's light,
 * Sec. 8): an equirectangular RGB map [H][W][3]; NULL clears it. */
void oracle_scene_set_environment(oscene* S, const float* env, int W, int H)
{
    free(S->env);
    S->env = NULL;
    S->env_w = S->env_h = 0;
    if (!env || W <= 0 || H <= 0) return;
    S->env = (double*)malloc(sizeof(double) * 3 * (size_t)W * (size_t)H);
    for (size_t i = 0; i < 3 * (size_t)W * (size_t)H; ++i) S->env[i] = env[i];
    S->env_w = W;
    S->env_h = H;
}

/* Radiance of the environment in unit direction d: longitude
 * u = atan2(d.x, -d.z) / 2pi + 1/2, colatitude v = acos(d.y) / pi, texel
 * (i, j) centred at ((i + 1/2) / W, (j + 1/2) / H); bilinear, wrapping in u
 * and clamping in v. */
static void env_lookup(const oscene* S, const double d[3], double L[3])
{
    L[0] = L[1] = L[2] = 0.0;
    if (!S->env) return;
    const int W = S->env_w, H = S->env_h;
    double dl = norm3(d);
    double y = d[1] / dl;
    if (y > 1.0) y = 1.0;
    if (y < -1.0) y = -1.0;
    double u = atan2(d[0] / dl, -d[2] / dl) / (2.0 * OPI) + 0.5;
    double v = acos(y) / OPI;
    double fx = u * W - 0.5, fy = v * H - 0.5;
    double i0f = floor(fx), j0f = floor(fy);
    double tx = fx - i0f, ty = fy - j0f;
    int i0 = (int)i0f, j0 = (int)j0f;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            int i = ((i0 + di) % W + W) % W;
            int j = j0 + dj;
            if (j < 0) j = 0;
            if (j > H - 1) j = H - 1;
            double w = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty);
            for (int c = 0; c < 3; ++c) L[c] += w * S->env[3 * ((size_t)j * W + i) + c];
        }
}

/* Environment radiance for n unit directions (rows of dirs) -> out [n][3]. */
void oracle_env_lookup(const oscene* S, const double* dirs, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) env_lookup(S, dirs + 3 * i, out + 3 * i);
}

void oracle_scene_info(const oscene* S, double* lo, double* hi, double* eps, double* L)
{
    for (int a = 0; a < 3; ++a) { lo[a] = S->slo[a]; hi[a] = S->shi[a]; }
    *eps = S->eps;
    *L = S->L;
}

/* ------------------------------------------------------------------ */
/* Closest hit                                                          */
/* ------------------------------------------------------------------ */
/* Line through o with direction d against the triangle's plane
 * (Moeller-Trumbore in FP64).  Returns 0 when the ray is parallel to the
 * plane.  lam = barycentric coordinates (weights of v0, v1, v2), cosabs =
 * |cos| of the angle between d and the face normal. */
static int tri_plane(const otri* tr, const double o[3], const double d[3],
                     double* t, double lam[3], double* cosabs)
{
    double p[3], s[3], q[3];
    cross3(d, tr->e2, p);
    double det = dot3(tr->e1, p);
    if (det == 0.0 || tr->area2 == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, tr->v0, s);
    double u = dot3(s, p) * inv;
    cross3(s, tr->e1, q);
    double v = dot3(d, q) * inv;
    *t = dot3(tr->e2, q) * inv;
    lam[0] = 1.0 - u - v; lam[1] = u; lam[2] = v;
    *cosabs = fabs(dot3(d, tr->ng)) / (norm3(d) * tr->area2);
    return 1;
}

/* One hit: triangle id (-1 = miss), distance, whether the ray meets the
 * front face (d . n_g < 0), and whether that facing is within rounding of
 * grazing (so a float32 evaluation may decide it either way). */
typedef struct { int32_t id; double t; int front; int front_amb; } ohit;

#define OMAXC 24
typedef struct {
    ohit nominal;        /* exact FP64 closest hit, ties by (t, id) */
    int n;               /* candidates: hits a perturbed ray may report */
    ohit c[OMAXC];
    int miss_possible;   /* a perturbed ray may miss everything */
    int overflow;        /* more candidates than OMAXC */
} ocands;

/* eta == 0: exact closest hit only.  eta > 0: additionally collect every
 * triangle that a ray perturbed by about eta * (L + t) could report as its
 * closest hit (see the header of oracle.py for the rule). */
static void closest(const oscene* S, const double o[3], const double d[3], int32_t skip,
                    double eta, ocands* out)
{
    out->nominal.id = -1; out->nominal.t = INFINITY; out->nominal.front = 0; out->nominal.front_amb = 0;
    out->n = 0; out->miss_possible = 1; out->overflow = 0;
    if (S->T == 0) return;
    double inv[3];
    for (int a = 0; a < 3; ++a) inv[a] = 1.0 / d[a];   /* +-inf for zero components */
    const double dl = norm3(d);
    const double mmax = eta * (S->L + S->diag);
    const double pad = (eta > 0 ? 20.0 * mmax : 0.0) + 1e-9 * (S->L + 1.0);
    double tc = INFINITY;      /* closest certain hit */
    double bound = INFINITY;   /* no triangle beyond this can matter */
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const onode* nd = &S->node[stack[--sp]];
        /* slab test against the padded box */
        double t0 = -pad / (dl > 0 ? dl : 1.0), t1 = bound + pad;
        int miss = 0;
        for (int a = 0; a < 3; ++a) {
            double lo = nd->lo[a] - pad, hi = nd->hi[a] + pad;
            if (d[a] == 0.0) {
                if (o[a] < lo || o[a] > hi) { miss = 1; break; }
                continue;
            }
            double ta = (lo - o[a]) * inv[a], tb = (hi - o[a]) * inv[a];
            if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
            if (t0 > t1) { miss = 1; break; }
        }
        if (miss) continue;
        if (nd->count == 0) {
            stack[sp++] = nd->left;
            stack[sp++] = nd->right;
            continue;
        }
        for (int k = nd->start; k < nd->start + nd->count; ++k) {
            int id = S->idx[k];
            if (id == skip) continue;
            const otri* tr = &S->tri[id];
            double t, lam[3], ca;
            if (!tri_plane(tr, o, d, &t, lam, &ca)) continue;
            int front = dot3(d, tr->ng) < 0.0;
            /* exact hit: inclusive edges, t > 0 */
            if (lam[0] >= 0 && lam[1] >= 0 && lam[2] >= 0 && t > 0) {
                if (t < out->nominal.t || (t == out->nominal.t && id < out->nominal.id)) {
                    out->nominal.id = id; out->nominal.t = t; out->nominal.front = front;
                }
            }
            if (eta <= 0) continue;
            double m = eta * (S->L + fabs(t));
            double mp = m / (ca > 0.05 ? ca : 0.05);
            int inflated = t > -m, certain = t > m;
            for (int i = 0; i < 3; ++i) {
                double dist = lam[i] * tr->h[i];
                if (dist < -mp) inflated = 0;
                if (dist < mp) certain = 0;
            }
            if (!inflated) continue;
            if (certain && t < tc) {
                tc = t;
                bound = tc + eta * (S->L + tc);
            }
            if (out->n < OMAXC) {
                ohit* h = &out->c[out->n++];
                h->id = id; h->t = t; h->front = front;
                h->front_amb = ca < 1e-5;
            } else {
                out->overflow = 1;
            }
        }
    }
    if (eta <= 0) { out->n = 0; out->miss_possible = out->nominal.id < 0; return; }
    /* keep inflated hits that are not beyond the certain closest hit */
    int w = 0;
    for (int i = 0; i < out->n; ++i)
        if (out->c[i].t <= bound) out->c[w++] = out->c[i];
    out->n = w;
    out->miss_possible = (tc == INFINITY);
    if (out->nominal.id >= 0) {
        const otri* tr = &S->tri[out->nominal.id];
        out->nominal.front_amb = fabs(dot3(d, tr->ng)) / (dl * tr->area2) < 1e-5;
    }
}

/* Brute-force closest hit over every triangle (exact FP64, ties by id). */
static void closest_brute(const oscene* S, const double o[3], const double d[3], int32_t skip, ohit* h)
{
    h->id = -1; h->t = INFINITY; h->front = 0; h->front_amb = 0;
    for (int64_t id = 0; id < S->T; ++id) {
        if (id == skip) continue;
        const otri* tr = &S->tri[id];
        double t, lam[3], ca;
        if (!tri_plane(tr, o, d, &t, lam, &ca)) continue;
        if (lam[0] >= 0 && lam[1] >= 0 && lam[2] >= 0 && t > 0) {
            if (t < h->t || (t == h->t && id < h->id)) {
                h->id = (int32_t)id; h->t = t; h->front = dot3(d, tr->ng) < 0.0;
            }
        }
    }
}

/* Public closest-hit query.  brute != 0 uses the brute-force loop (exact
 * hit only; candidates left empty).  cand_* are nR x OMAXC. */
int oracle_closest(const oscene* S, const double* orig, const double* dir, int64_t nR,
                   const int32_t* skip, double eta, int brute,
                   int32_t* hit_id, double* hit_t, int32_t* hit_front,
                   int32_t* cand_id, double* cand_t, int32_t* n_cand,
                   int32_t* miss_possible)
{
    for (int64_t r = 0; r < nR; ++r) {
        const double* o = orig + 3 * r;
        const double* d = dir + 3 * r;
        int32_t sk = skip ? skip[r] : -1;
        if (brute) {
            ohit h;
            closest_brute(S, o, d, sk, &h);
            hit_id[r] = h.id; hit_t[r] = h.t; hit_front[r] = h.front;
            if (n_cand) n_cand[r] = 0;
            if (miss_possible) miss_possible[r] = h.id < 0;
            continue;
        }
        ocands c;
        closest(S, o, d, sk, eta, &c);
        hit_id[r] = c.nominal.id; hit_t[r] = c.nominal.t; hit_front[r] = c.nominal.front;
        if (n_cand) n_cand[r] = c.overflow ? -1 : c.n;
        if (miss_possible) miss_possible[r] = c.miss_possible;
        if (cand_id)
            for (int i = 0; i < c.n; ++i) { cand_id[OMAXC*r+i] = c.c[i].id; cand_t[OMAXC*r+i] = c.c[i].t; }
    }
    return OMAXC;
}

/* ------------------------------------------------------------------ */
/* Sampling (Sec. 6: BRDF importance sampling in stage 1)               */
/* ------------------------------------------------------------------ */
/* Orthonormal basis (t, b, n) around a unit normal: Duff et al.,
 * "Building an orthonormal basis, revisited", JCGT 2017.  The branch is
 * taken at n.z >= -1e-6 (the float constant), not at the sign of n.z, so
 * that faces with n.z = 0 -- axis-aligned walls, symmetric sphere facets,
 * whose computed z is +-0 or a rounding-sized value of either sign -- get
 * the same frame on every side. */
#define OR_ONB_BRANCH ((double)(-1e-6f))
static void onb(const double n[3], double t[3], double b[3])
{
    double s = n[2] >= OR_ONB_BRANCH ? 1.0 : -1.0;
    double a = -1.0 / (s + n[2]);
    double c = n[0] * n[1] * a;
    t[0] = 1.0 + s * n[0] * n[0] * a; t[1] = s * c; t[2] = -s * n[0];
    b[0] = c; b[1] = s + n[1] * n[1] * a; b[2] = -n[1];
}

static void to_world(const double t[3], const double b[3], const double n[3],
                     double x, double y, double z, double w[3])
{
    for (int a = 0; a < 3; ++a) w[a] = x * t[a] + y * b[a] + z * n[a];
}

/* Smith-GGX masking for one direction with cosine mu to the normal
 * (Walter et al. 2007, separable form), alpha2 = alpha^2. */
static double smith_g1(double mu, double alpha2)
{
    return 2.0 * mu / (mu + sqrt(alpha2 + (1.0 - alpha2) * mu * mu));
}

/* ------------------------------------------------------------------ */
/* Bake (Eq. 6, 7, 9)                                                   */
/* ------------------------------------------------------------------ */
typedef struct {
    const oscene* S;
    const float *qx, *qn, *qwo;
    const int32_t* qtri;
    int64_t N;
    uint64_t seed;
    uint32_t request_id, point_base;
    int spp_d, spp_s, K;
    const double* sigma;
    double eta;
    double *nominal, *lo, *hi;
    int64_t* n_amb;
    int64_t next;      /* work counter */
} bake_job;

/* Incident radiance for one hit: emission counted on the front face only,
 * plus the per-triangle cache; a miss brings nothing. */
/* Incident radiance along d from a hit on triangle id at distance t from
 * o: front-face emission + the cache L' there (Eq. 9); a miss brings the
 * environment (or 0). */
static void radiance(const oscene* S, int32_t id, int front, const double o[3], const double d[3],
                     double t, double L[3])
{
    if (id < 0) { env_lookup(S, d, L); return; }
    double p[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]}, C[3];
    cache_at(S, id, p, C);
    for (int a = 0; a < 3; ++a) L[a] = (front ? S->Le[3*id+a] : 0.0) + C[a];
}

/* Cache values of every voxel a float32 hit point near p may fall in:
 * the cell of p and its neighbours across faces within w (a fraction of
 * the cell) of p. */
static void voxel_range_w(const oscene* S, const double p[3], double w, double lo[3], double hi[3]);
static void voxel_range(const oscene* S, const double p[3], double lo[3], double hi[3])
{
    voxel_range_w(S, p, 1e-3, lo, hi);
}
static void voxel_range_w(const oscene* S, const double p[3], double w, double lo[3], double hi[3])
{
    const int R = S->vox_r;
    double fr[3];
    int64_t v = voxel_of(S, R, p, fr);
    int64_t base[3] = {v % R, (v / R) % R, v / ((int64_t)R * R)};
    for (int c = 0; c < 3; ++c) { lo[c] = INFINITY; hi[c] = -INFINITY; }
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int dd[3] = {dx, dy, dz};
                int ok = 1;
                int64_t ix[3];
                for (int a = 0; a < 3; ++a) {
                    if (dd[a] == -1 && !(fr[a] < w)) ok = 0;
                    if (dd[a] == 1 && !(fr[a] > 1.0 - w)) ok = 0;
                    ix[a] = base[a] + dd[a];
                    if (ix[a] < 0 || ix[a] > R - 1) ok = 0;
                }
                if (!ok) continue;
                int64_t w = (ix[2] * R + ix[1]) * R + ix[0];
                for (int c = 0; c < 3; ++c) {
                    if (S->vox[4*w+c] < lo[c]) lo[c] = S->vox[4*w+c];
                    if (S->vox[4*w+c] > hi[c]) hi[c] = S->vox[4*w+c];
                }
            }
}

/* Range of the incident radiance over every hit a perturbed ray may report
 * (candidates, both facings when grazing, and a miss when possible). */
static int radiance_range(const oscene* S, const ocands* c, const double o[3], const double d[3],
                          double Lmin[3], double Lmax[3])
{
    for (int a = 0; a < 3; ++a) { Lmin[a] = INFINITY; Lmax[a] = -INFINITY; }
    int alts = 0;
    double L[3];
#define OR_ACC(id_, fr_, t_) do { radiance(S, (id_), (fr_), o, d, (t_), L); ++alts; \
        for (int a = 0; a < 3; ++a) { if (L[a] < Lmin[a]) Lmin[a] = L[a]; if (L[a] > Lmax[a]) Lmax[a] = L[a]; } \
        if ((id_) >= 0 && S->vox) { \
            double p_[3] = {o[0] + (t_) * d[0], o[1] + (t_) * d[1], o[2] + (t_) * d[2]}, vl[3], vh[3]; \
            voxel_range(S, p_, vl, vh); \
            for (int a = 0; a < 3; ++a) { double e_ = (fr_) ? S->Le[3*(id_)+a] : 0.0; \
                Lmin[a] = fmin(Lmin[a], e_ + vl[a]); \
                Lmax[a] = fmax(Lmax[a], e_ + vh[a]); } } \
    } while (0)
    OR_ACC(c->nominal.id, c->nominal.front, c->nominal.t);
    if (c->nominal.id >= 0 && c->nominal.front_amb) OR_ACC(c->nominal.id, !c->nominal.front, c->nominal.t);
    for (int i = 0; i < c->n; ++i) {
        OR_ACC(c->c[i].id, c->c[i].front, c->c[i].t);
        if (c->c[i].front_amb) OR_ACC(c->c[i].id, !c->c[i].front, c->c[i].t);
    }
    if (c->miss_possible) OR_ACC(-1, 0, 0.0);
#undef OR_ACC
    int amb = 0;
    for (int a = 0; a < 3; ++a) if (Lmin[a] != Lmax[a]) amb = 1;
    if (c->overflow) {
        /* Too many candidates to enumerate: bound by every value in the scene. */
        for (int a = 0; a < 3; ++a) { Lmin[a] = 0.0; Lmax[a] = INFINITY; }
        amb = 1;
    }
    return amb;
}

static void bake_point(bake_job* J, int64_t p)
{
    const oscene* S = J->S;
    const int K = J->K;
    const int W = 3 + 6 * K;
    double* nom = J->nominal + (size_t)W * p;
    double* lo = J->lo ? J->lo + (size_t)W * p : NULL;
    double* hi = J->hi ? J->hi + (size_t)W * p : NULL;
    int64_t amb_rays = 0;
    for (int i = 0; i < W; ++i) { nom[i] = 0.0; if (lo) lo[i] = 0.0; if (hi) hi[i] = 0.0; }

    double x[3], n[3], wo[3];
    for (int a = 0; a < 3; ++a) { x[a] = J->qx[3*p+a]; n[a] = J->qn[3*p+a]; wo[a] = J->qwo[3*p+a]; }
    normalize3(n);
    normalize3(wo);
    const int32_t skip = J->qtri[p];
    double o[3];
    for (int a = 0; a < 3; ++a) o[a] = x[a] + S->eps * n[a];
    double tb[3], bb[3];
    onb(n, tb, bb);
    const double mu_o = dot3(n, wo);
    const uint32_t key[2] = {(uint32_t)J->seed, (uint32_t)(J->seed >> 32)};
    const uint32_t pid = J->point_base + (uint32_t)p;

    /* Diffuse shading L_d (Eq. 6): cosine-weighted directions, pdf = cos/pi,
     * so each sample contributes its incident radiance unweighted. */
    for (int s = 0; s < J->spp_d; ++s) {
        uint32_t ctr[4] = {pid, (uint32_t)s, 0u, J->request_id}, r[4];
        philox10(ctr, key, r);
        double u1 = u24(r[0]), u2 = u24(r[1]);
        strat_uv((uint32_t)s, J->spp_d, &u1, &u2);
        double rad = sqrt(u1), phi = 2.0 * OPI * u2;
        double wi[3];
        to_world(tb, bb, n, rad * cos(phi), rad * sin(phi), sqrt(1.0 - u1), wi);
        ocands c;
        closest(S, o, wi, skip, J->eta, &c);
        double L[3];
        radiance(S, c.nominal.id, c.nominal.front, o, wi, c.nominal.t, L);
        for (int a = 0; a < 3; ++a) nom[a] += L[a];
        if (lo) {
            double Lmin[3], Lmax[3];
            amb_rays += radiance_range(S, &c, o, wi, Lmin, Lmax);
            for (int a = 0; a < 3; ++a) { lo[a] += Lmin[a]; hi[a] += Lmax[a]; }
        }
    }
    for (int a = 0; a < 3; ++a) {
        nom[a] /= J->spp_d;
        if (lo) { lo[a] /= J->spp_d; hi[a] /= J->spp_d; }
    }

    /* Specular shadings L_s0, L_s1 (Eq. 6, 7) per roughness level: GGX
     * half-vector sampling with density D(h)(n.h) (Walter et al. 2007),
     * reflected to wi; the estimator weight F*D*G/(4 n.wo) / pdf(wi) reduces
     * to F * G * (wo.h) / ((n.wo)(n.h)).  Points seen at n.wo <= 1e-2 get 0. */
    if (mu_o <= 1e-2) goto done;
    for (int k = 0; k < K; ++k) {
        const double alpha = J->sigma[k] * J->sigma[k];
        const double a2 = alpha * alpha;
        const double g1o = smith_g1(mu_o, a2);
        double s0[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
        double l0[3] = {0, 0, 0}, l1[3] = {0, 0, 0}, h0[3] = {0, 0, 0}, h1[3] = {0, 0, 0};
        for (int s = 0; s < J->spp_s; ++s) {
            uint32_t ctr[4] = {pid, (uint32_t)s, (uint32_t)(k + 1), J->request_id}, r[4];
            philox10(ctr, key, r);
            double u1 = u24(r[0]), u2 = u24(r[1]);
            strat_uv((uint32_t)s, J->spp_s, &u1, &u2);
            double cos2 = (1.0 - u1) / (1.0 + (a2 - 1.0) * u1);
            double ch = sqrt(cos2), sh = sqrt(fmax(0.0, 1.0 - cos2));
            double phi = 2.0 * OPI * u2;
            double h[3];
            to_world(tb, bb, n, sh * cos(phi), sh * sin(phi), ch, h);
            double c = dot3(wo, h);
            double wi[3];
            for (int a = 0; a < 3; ++a) wi[a] = 2.0 * c * h[a] - wo[a];
            double mu_i = dot3(n, wi);
            if (mu_i <= 0.0 || c <= 0.0) continue;     /* counts as a zero sample */
            double G = smith_g1(mu_i, a2) * g1o;
            double w = G * c / (mu_o * ch);
            double F1 = pow(1.0 - c, 5.0);
            double F0 = 1.0 - F1;
            ocands cd;
            closest(S, o, wi, skip, J->eta, &cd);
            double L[3];
            radiance(S, cd.nominal.id, cd.nominal.front, o, wi, cd.nominal.t, L);
            for (int a = 0; a < 3; ++a) { s0[a] += L[a] * F0 * w; s1[a] += L[a] * F1 * w; }
            if (lo) {
                double Lmin[3], Lmax[3];
                amb_rays += radiance_range(S, &cd, o, wi, Lmin, Lmax);
                for (int a = 0; a < 3; ++a) {
                    l0[a] += Lmin[a] * F0 * w; h0[a] += Lmax[a] * F0 * w;
                    l1[a] += Lmin[a] * F1 * w; h1[a] += Lmax[a] * F1 * w;
                }
            }
        }
        for (int a = 0; a < 3; ++a) {
            nom[3 + 3*k + a] = s0[a] / J->spp_s;
            nom[3 + 3*K + 3*k + a] = s1[a] / J->spp_s;
            if (lo) {
                lo[3 + 3*k + a] = l0[a] / J->spp_s;  hi[3 + 3*k + a] = h0[a] / J->spp_s;
                lo[3 + 3*K + 3*k + a] = l1[a] / J->spp_s;  hi[3 + 3*K + 3*k + a] = h1[a] / J->spp_s;
            }
        }
    }
done:
    if (J->n_amb) J->n_amb[p] = amb_rays;
}

static void* bake_worker(void* arg)
{
    bake_job* J = (bake_job*)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (p >= J->N) break;
        bake_point(J, p);
    }
    return NULL;
}

/* Bake every query point.  Output row per point (length 3 + 6K):
 *   [L_d rgb | L_s0(sigma_0..K-1) rgb | L_s1(sigma_0..K-1) rgb].
 * nominal: the estimator on exact FP64 hits.  lo / hi (nullable, need
 * eta > 0): the same estimator with every ray's incident radiance replaced
 * by its minimum / maximum over the hits a perturbed ray may report.
 * n_amb (nullable): per point, the number of rays with more than one
 * possible radiance. */
int oracle_bake(const oscene* S, const float* qx, const float* qn, const float* qwo,
                const int32_t* qtri, int64_t N, uint64_t seed, uint32_t request_id,
                uint32_t point_base, int spp_d, int spp_s, int K, const double* sigma,
                double eta, int nthreads, double* nominal, double* lo, double* hi,
                int64_t* n_amb)
{
    bake_job J;
    J.S = S; J.qx = qx; J.qn = qn; J.qwo = qwo; J.qtri = qtri; J.N = N;
    J.seed = seed; J.request_id = request_id; J.point_base = point_base;
    J.spp_d = spp_d; J.spp_s = spp_s; J.K = K; J.sigma = sigma; J.eta = eta;
    J.nominal = nominal; J.lo = (eta > 0) ? lo : NULL; J.hi = (eta > 0) ? hi : NULL;
    J.n_amb = n_amb; J.next = 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, bake_worker, &J);
    bake_worker(&J);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Pinhole first hits (query generation)                                */
/* ------------------------------------------------------------------ */
/* Camera row: eye xyz, forward xyz, up xyz, vertical fov (radians).
 * right = normalize(fwd x up), up' = right x fwd; pixel (i, j) of a W x H
 * image (j = 0 at the top) looks along
 *   normalize(fwd + sx * right + sy * up'),
 *   sx = (2 (i + 0.5) / W - 1) * tan(fov/2) * W / H,
 *   sy = (1 - 2 (j + 0.5) / H) * tan(fov/2).
 * Output per pixel p (view-major, then row, then column): query record
 * x = eye + t d, n = unit face normal turned toward the camera, wo = -d,
 * tri = hit triangle, valid = hit; plus the candidate count as in
 * oracle_closest (n_cand = number of alternative hits, miss_possible). */
int oracle_camera_queries(const oscene* S, const float* cams, int n_views, int W, int H,
                          const int64_t* pixels, int64_t n_pix, double eta,
                          double* qx, double* qn, double* qwo, int32_t* qtri,
                          int32_t* n_cand, int32_t* cand_id, int32_t* miss_possible)
{
    for (int64_t k = 0; k < n_pix; ++k) {
        int64_t p = pixels[k];
        int v = (int)(p / ((int64_t)W * H));
        if (v < 0 || v >= n_views) return -1;
        int64_t rem = p % ((int64_t)W * H);
        int j = (int)(rem / W), i = (int)(rem % W);
        const float* c = cams + 10 * v;
        double eye[3] = {c[0], c[1], c[2]}, fwd[3] = {c[3], c[4], c[5]}, up[3] = {c[6], c[7], c[8]};
        normalize3(fwd);
        double right[3], up2[3];
        cross3(fwd, up, right); normalize3(right);
        cross3(right, fwd, up2);
        double th = tan(0.5 * (double)c[9]);
        double sx = (2.0 * (i + 0.5) / W - 1.0) * th * ((double)W / H);
        double sy = (1.0 - 2.0 * (j + 0.5) / H) * th;
        double d[3];
        for (int a = 0; a < 3; ++a) d[a] = fwd[a] + sx * right[a] + sy * up2[a];
        normalize3(d);
        ocands cd;
        closest(S, eye, d, -1, eta, &cd);
        qtri[k] = cd.nominal.id;
        if (n_cand) n_cand[k] = cd.overflow ? -1 : cd.n;
        if (miss_possible) miss_possible[k] = cd.miss_possible;
        if (cand_id) for (int q = 0; q < cd.n; ++q) cand_id[OMAXC * k + q] = cd.c[q].id;
        if (cd.nominal.id < 0) {
            for (int a = 0; a < 3; ++a) { qx[3*k+a] = 0; qn[3*k+a] = 0; qwo[3*k+a] = 0; }
            continue;
        }
        const otri* tr = &S->tri[cd.nominal.id];
        double ng[3] = {tr->ng[0], tr->ng[1], tr->ng[2]};
        normalize3(ng);
        double sgn = dot3(ng, d) > 0 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) {
            qx[3*k+a] = eye[a] + cd.nominal.t * d[a];
            qn[3*k+a] = sgn * ng[a];
            qwo[3*k+a] = -d[a];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Morton codes and the binary radix tree (bit-exact LBVH targets)      */
/* ------------------------------------------------------------------ */
/* Per triangle: box centre c = 0.5 * (double(min) + double(max)) per axis,
 * quantised against the scene box [lo, hi] taken from the float vertices:
 *   q = min(2^21 - 1, floor((c - lo) * (2^21 / (hi - lo))))   (q = 0 if hi == lo)
 * with every operation a single IEEE double rounding.  Bit i of qx, qy, qz
 * goes to bit 3i+2, 3i+1, 3i of the 63-bit code. */
static uint64_t spread21(uint32_t v)
{
    uint64_t r = 0;
    for (int i = 0; i < 21; ++i) r |= (uint64_t)((v >> i) & 1u) << (3 * i);
    return r;
}

int oracle_morton(const float* V, int64_t nV, const int32_t* F, int64_t T, uint64_t* codes)
{
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nV; ++i)
        for (int a = 0; a < 3; ++a) {
            if (V[3*i+a] < lo[a]) lo[a] = V[3*i+a];
            if (V[3*i+a] > hi[a]) hi[a] = V[3*i+a];
        }
    for (int64_t t = 0; t < T; ++t) {
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            float x0 = V[3*F[3*t+0]+a], x1 = V[3*F[3*t+1]+a], x2 = V[3*F[3*t+2]+a];
            float mn = x0 < x1 ? x0 : x1; mn = mn < x2 ? mn : x2;
            float mx = x0 > x1 ? x0 : x1; mx = mx > x2 ? mx : x2;
            double c = 0.5 * ((double)mn + (double)mx);
            double ext = (double)hi[a] - (double)lo[a];
            if (!(ext > 0.0)) { q[a] = 0; continue; }
            double scale = 2097152.0 / ext;
            double f = floor((c - (double)lo[a]) * scale);
            if (f < 0.0) f = 0.0;
            if (f > 2097151.0) f = 2097151.0;
            q[a] = (uint32_t)f;
        }
        codes[t] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
    }
    return 0;
}

/* Length of the common prefix of the augmented keys (code_i || i) and
 * (code_j || j): 64-bit code, then 32-bit index. */
static int prefix_len(const uint64_t* code, int64_t i, int64_t j)
{
    uint64_t x = code[i] ^ code[j];
    if (x) return __builtin_clzll(x);
    uint32_t y = (uint32_t)i ^ (uint32_t)j;
    return 64 + (y ? __builtin_clz(y) : 32);
}

/* bit at position `pos` counted from the top of the 96-bit augmented key */
static int key_bit(const uint64_t* code, int64_t i, int pos)
{
    if (pos < 64) return (int)((code[i] >> (63 - pos)) & 1u);
    return (int)(((uint32_t)i >> (31 - (pos - 64))) & 1u);
}

typedef struct {
    const uint64_t* code;
    const float* box;     /* T x 6 triangle boxes in sorted order: lo xyz, hi xyz */
    int32_t *first, *last, *split;
    float* nbox;          /* (T-1) x 6 */
    int64_t n;
} rt_job;

/* Radix-tree node over sorted keys [f, l], f < l: split after the last key
 * whose bit at the first differing position is 0.  Writes node boxes as the
 * float min / max over the triangles of the range (children first). */
static void rt_build(rt_job* R, int64_t f, int64_t l, float out_box[6])
{
    if (f == l) {
        for (int a = 0; a < 6; ++a) out_box[a] = R->box[6*f+a];
        return;
    }
    int64_t id = R->n++;
    int pos = prefix_len(R->code, f, l);
    int64_t s = f;
    while (s + 1 <= l && key_bit(R->code, s + 1, pos) == 0) ++s;
    R->first[id] = (int32_t)f; R->last[id] = (int32_t)l; R->split[id] = (int32_t)s;
    float bl[6], br[6];
    rt_build(R, f, s, bl);
    rt_build(R, s + 1, l, br);
    for (int a = 0; a < 3; ++a) {
        out_box[a] = bl[a] < br[a] ? bl[a] : br[a];
        out_box[3+a] = bl[3+a] > br[3+a] ? bl[3+a] : br[3+a];
    }
    for (int a = 0; a < 6; ++a) R->nbox[6*id+a] = out_box[a];
}

/* codes: sorted Morton codes (ties in index order); tri_box: T x 6 boxes of
 * the triangles in that order.  Output: T-1 internal nodes in pre-order. */
int oracle_radix_tree(const uint64_t* codes, const float* tri_box, int64_t T,
                      int32_t* first, int32_t* last, int32_t* split, float* node_box)
{
    if (T < 2) return 0;
    rt_job R = {codes, tri_box, first, last, split, node_box, 0};
    float root[6];
    rt_build(&R, 0, T - 1, root);
    return (int)R.n;
}

/* ------------------------------------------------------------------ */
/* Stage-3 path-traced refinement (Sec. 4.3, Eq. 10; MIS per Sec. 6)    */
/* ------------------------------------------------------------------ */
/* A sample starts like the stage-1 bake (same lobe, same Philox stream)
 * and grows its path through surfaces with roughness <= sigma_c, sampling
 * the full BRDF of Eq. 1 there, until it reaches an emitter (radiance
 * L_e, front face only) or a surface rougher than sigma_c (radiance L',
 * the diffuse cache).  With mis != 0 every vertex also samples a point on
 * the emitters (area-uniform over all emitter triangles) and the two
 * strategies are combined with the power heuristic (Veach 1997).
 *
 * Philox counters (lobe as in the bake: 0 diffuse, k+1 roughness level k):
 *   lobe direction at x          (pid, s, lobe, rid)                 words 0, 1
 *   emitter sample at x          (pid, s, lobe | 0x100, rid)         words 0 (triangle), 1, 2 (point)
 *   BRDF at path vertex i >= 1   (pid, s, lobe | i << 9, rid)        words 0, 1 (direction), 2 (lobe)
 *   emitter sample at vertex i   (pid, s, lobe | i << 9 | 0x100, rid) words 0, 1, 2
 * Path vertices beyond the first hit are at most max_depth.  Per-vertex
 * choice of the diffuse lobe: P_d = clamp(mean(k_d) / (mean(k_d) +
 * mean(k_s)), 0.1, 0.9); at vertices seen at n.wo <= 1e-2 the specular lobe
 * is dropped (P_d = 1), as in the bake. */
typedef struct {
    const oscene* S;
    const float *ma, *ms, *mm;   /* per-triangle albedo [T,3], roughness, metallic */
    int n_emit;
    int* emit;                   /* emitter triangles in index order */
    double* cdf;                 /* cumulative areas */
    double A;                    /* total emitter area */
    const float *qx, *qn, *qwo;
    const int32_t* qtri;
    int64_t N;
    uint64_t seed;
    uint32_t request_id, point_base;
    int spp_d, spp_s, K;
    const double* sigma;
    double sigma_c;
    int max_depth, mis;
    double eta;
    double* out;                 /* N x (3 + 6K) */
    double* per_sample;          /* nullable: N x (1+K) x Smax x 6 */
    uint8_t* amb;                /* nullable: N x (1+K) x Smax */
    double *ps_lo, *ps_hi;       /* nullable: N x (1+K) x Smax x 6, ranges (see sample_range) */
    uint8_t* unb;                /* nullable: N x (1+K) x Smax, 1 = range not bounded */
    int smax;
    int64_t next;
} refine_job;

static double ggx_D(double ch, double a2)
{
    double c2 = ch * ch;
    double den = (1.0 - c2) + a2 * c2;
    return a2 / (OPI * den * den);
}

static void philox_words(uint32_t pid, uint32_t s, uint32_t lane, uint32_t rid, uint64_t seed, double u[4])
{
    uint32_t ctr[4] = {pid, s, lane, rid}, key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)}, r[4];
    philox10(ctr, key, r);
    for (int i = 0; i < 4; ++i) u[i] = u24(r[i]);
}

/* Emitter sample: triangle by area (first k with cdf[k] > u0 A), uniform
 * point by the square-root map.  Returns the triangle; *amb when u0 A lies
 * within 1e-6 A of a cumulative boundary. */
static int emitter_sample(const refine_job* R, const double u[4], double y[3], int* amb)
{
    double target = u[0] * R->A;
    int lo = 0, hi = R->n_emit - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (R->cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    if (R->n_emit > 1) {
        if (fabs(R->cdf[lo] - target) < 1e-6 * R->A) *amb = 1;
        if (lo > 0 && fabs(R->cdf[lo - 1] - target) < 1e-6 * R->A) *amb = 1;
    }
    const otri* tr = &R->S->tri[R->emit[lo]];
    double r1 = sqrt(u[1]);
    double b0 = 1.0 - r1, b1 = r1 * (1.0 - u[2]), b2 = r1 * u[2];
    for (int a = 0; a < 3; ++a) y[a] = b0 * tr->v0[a] + b1 * tr->v1[a] + b2 * tr->v2[a];
    return R->emit[lo];
}

static int is_emitter(const oscene* S, int t)
{
    return S->Le[3*t] > 0 || S->Le[3*t+1] > 0 || S->Le[3*t+2] > 0;
}

/* Closest hit with ambiguity flag (candidate set larger than one, or a
 * grazing facing, or a possible miss next to a hit). */
static void trace_flag(const refine_job* R, const double o[3], const double d[3], int skip,
                       ohit* h, int* amb)
{
    ocands c;
    closest(R->S, o, d, skip, R->eta, &c);
    *h = c.nominal;
    if (R->eta > 0) {
        int distinct = 0;
        for (int i = 0; i < c.n; ++i) if (c.c[i].id != c.nominal.id) distinct = 1;
        if (distinct || c.overflow || c.nominal.front_amb || (c.miss_possible && c.nominal.id >= 0) ||
            (!c.miss_possible && c.nominal.id < 0))
            *amb = 1;
        for (int i = 0; i < c.n; ++i) if (c.c[i].front_amb) *amb = 1;
    }
}

/* Probability of drawing the diffuse lobe at a vertex of triangle t. */
static double vertex_pd(const refine_job* R, int t, double mu_o)
{
    double kd = 0, ks = 0;
    const double m = R->mm[t];
    for (int c = 0; c < 3; ++c) {
        kd += R->ma[3*t+c] * (1.0 - m);
        ks += 0.04 * (1.0 - m) + R->ma[3*t+c] * m;
    }
    double Pd = kd / (kd + ks);
    if (Pd < 0.1) Pd = 0.1;
    if (Pd > 0.9) Pd = 0.9;
    return mu_o > 1e-2 ? Pd : 1.0;
}

/* Full BRDF of Eq. 1 (including the cosine) at a vertex, RGB, and the pdf
 * of the vertex's mixture sampler; P_d as in the header. */
/* Relative change of the GGX distribution per radian of half-vector tilt,
 * |d ln D / d theta| = 4 tan / (tan^2 + alpha^2) (up to 1 - alpha^2). */
static double ggx_log_slope(double ch, double sh, double a2)
{
    if (ch <= 0) return INFINITY;
    double t = sh / ch;
    return 4.0 * t / (t * t + a2);
}

/* A half vector recomputed from two directions carries float32 rounding of
 * about 2e-6 rad on the kernel's side; where D changes by more than 1e-4
 * under that tilt the sample is flagged as ill-conditioned. */
#define OR_SLOPE_LIMIT 50.0

static void vertex_brdf_h(const refine_job* R, int t, const double n[3], const double wo[3],
                          const double wi[3], const double* hs, double f[3], double* pdf,
                          double* Pd_out, int* amb);

static void vertex_brdf(const refine_job* R, int t, const double n[3], const double wo[3],
                        const double wi[3], double f[3], double* pdf, double* Pd_out, int* amb)
{
    vertex_brdf_h(R, t, n, wo, wi, NULL, f, pdf, Pd_out, amb);
}

/* hs != NULL: wi was reflected about the sampled half vector hs, whose D is
 * then evaluated at hs itself (no recomputation from wi). */
static void vertex_brdf_h(const refine_job* R, int t, const double n[3], const double wo[3],
                          const double wi[3], const double* hs, double f[3], double* pdf,
                          double* Pd_out, int* amb)
{
    const double a[3] = {R->ma[3*t], R->ma[3*t+1], R->ma[3*t+2]};
    const double sg = R->ms[t], m = R->mm[t];
    const double al = sg * sg, a2 = al * al;
    double kd[3], ks[3];
    for (int c = 0; c < 3; ++c) { kd[c] = a[c] * (1.0 - m); ks[c] = 0.04 * (1.0 - m) + a[c] * m; }
    const double mu_o = dot3(n, wo), mu_i = dot3(n, wi);
    double Pd = vertex_pd(R, t, mu_o);
    const int spec = mu_o > 1e-2;
    if (fabs(mu_o - 1e-2) < 1e-6) *amb = 1;
    *Pd_out = Pd;
    for (int c = 0; c < 3; ++c) f[c] = 0.0;
    *pdf = 0.0;
    if (fabs(mu_i) < 1e-5) *amb = 1;
    if (mu_i <= 0.0) return;
    for (int c = 0; c < 3; ++c) f[c] = kd[c] * mu_i / OPI;
    *pdf = Pd * mu_i / OPI;
    if (!spec) return;
    double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
    if (hs) { h[0] = hs[0]; h[1] = hs[1]; h[2] = hs[2]; }
    normalize3(h);
    const double ch = dot3(n, h), co = dot3(wo, h);
    if (fabs(co) < 1e-5) *amb = 1;
    if (ch <= 0.0 || co <= 0.0) return;
    const double D = ggx_D(ch, a2);
    if (!hs) {
        double cr[3];
        cross3(n, h, cr);
        if (ggx_log_slope(ch, norm3(cr), a2) > OR_SLOPE_LIMIT) *amb = 1;
    }
    const double G = smith_g1(mu_i, a2) * smith_g1(mu_o, a2);
    const double F1 = pow(1.0 - co, 5.0), F0 = 1.0 - F1;
    for (int c = 0; c < 3; ++c) f[c] += (ks[c] * F0 + F1) * D * G / (4.0 * mu_o);
    *pdf += (1.0 - Pd) * D * ch / (4.0 * co);
}

/* Radiance arriving along a path that leaves `o` (offset origin of a
 * surface point on triangle `skip`) in direction d, estimated from the
 * first hit on (Eq. 10 with MIS).  pdf_prev = density with which d was
 * drawn (for the MIS weight of an emitter hit). */
static void path_radiance(const refine_job* R, const double o0[3], const double d0[3], int skip0,
                          double pdf_prev, uint32_t pid, uint32_t s, uint32_t lobe, double L[3],
                          int* amb)
{
    const oscene* S = R->S;
    double o[3] = {o0[0], o0[1], o0[2]}, d[3] = {d0[0], d0[1], d0[2]};
    int skip = skip0;
    double beta[3] = {1, 1, 1};
    L[0] = L[1] = L[2] = 0.0;
    for (int depth = 1;; ++depth) {
        ohit h;
        trace_flag(R, o, d, skip, &h, amb);
        if (h.id < 0) {
            double Le[3];
            env_lookup(S, d, Le);
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * Le[c];
            return;
        }
        if (is_emitter(S, h.id)) {
            if (!h.front) return;
            double w = 1.0;
            if (R->mis && R->n_emit > 0) {
                const otri* tr = &S->tri[h.id];
                double ce = fabs(dot3(d, tr->ng)) / tr->area2;
                double pl = h.t * h.t / (R->A * ce);
                w = pdf_prev * pdf_prev / (pdf_prev * pdf_prev + pl * pl);
            }
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * w * S->Le[3*h.id+c];
            return;
        }
        if ((double)R->ms[h.id] > R->sigma_c) {
            double p[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]}, C[3];
            if (voxel_ambiguous(S, p)) *amb = 1;
            cache_at(S, h.id, p, C);
            for (int c = 0; c < 3; ++c) L[c] += beta[c] * C[c];
            return;
        }
        if (depth > R->max_depth) return;
        /* continue through a smooth surface */
        const otri* tr = &S->tri[h.id];
        double x[3], n[3] = {tr->ng[0], tr->ng[1], tr->ng[2]}, wo[3] = {-d[0], -d[1], -d[2]};
        normalize3(n);
        for (int a = 0; a < 3; ++a) x[a] = o[a] + h.t * d[a];
        if (dot3(n, wo) < 0) for (int a = 0; a < 3; ++a) n[a] = -n[a];
        if (fabs(n[2] - OR_ONB_BRANCH) < 2e-7) *amb = 1;    /* frame branch within rounding */
        double xo[3];
        for (int a = 0; a < 3; ++a) xo[a] = x[a] + S->eps * n[a];
        const uint32_t lane = lobe | ((uint32_t)depth << 9);
        if (R->mis && R->n_emit > 0) {      /* next-event estimation at this vertex */
            double u[4], y[3];
            philox_words(pid, s, lane | 0x100u, R->request_id, R->seed, u);
            int e = emitter_sample(R, u, y, amb);
            double wl[3];
            sub3(y, xo, wl);
            double dist = norm3(wl);
            for (int a = 0; a < 3; ++a) wl[a] /= dist;
            const otri* te = &S->tri[e];
            double ce = -dot3(wl, te->ng) / te->area2;
            if (fabs(ce) < 1e-5) *amb = 1;
            if (ce > 0) {
                double f[3], pb, Pd;
                vertex_brdf(R, h.id, n, wo, wl, f, &pb, &Pd, amb);
                if (f[0] > 0 || f[1] > 0 || f[2] > 0) {
                    ohit vh;
                    trace_flag(R, xo, wl, h.id, &vh, amb);
                    if (vh.id == e) {
                        double pl = dist * dist / (R->A * ce);
                        double w = pl * pl / (pl * pl + pb * pb);
                        for (int c = 0; c < 3; ++c) L[c] += beta[c] * w * S->Le[3*e+c] * f[c] / pl;
                    }
                }
            }
        }
        /* BRDF sample */
        double u[4];
        philox_words(pid, s, lane, R->request_id, R->seed, u);
        double Pd = vertex_pd(R, h.id, dot3(n, wo));
        double tb[3], bb[3], wi[3];
        onb(n, tb, bb);
        if (fabs(u[2] - Pd) < 1e-5) *amb = 1;
        double hh[3];
        const int glossy = !(u[2] < Pd);
        if (!glossy) {
            double rad = sqrt(u[0]), phi = 2.0 * OPI * u[1];
            to_world(tb, bb, n, rad * cos(phi), rad * sin(phi), sqrt(1.0 - u[0]), wi);
        } else {
            const double al = (double)R->ms[h.id] * (double)R->ms[h.id], a2 = al * al;
            double cos2 = (1.0 - u[0]) / (1.0 + (a2 - 1.0) * u[0]);
            double ch = sqrt(cos2), sh = sqrt(fmax(0.0, 1.0 - cos2)), phi = 2.0 * OPI * u[1];
            to_world(tb, bb, n, sh * cos(phi), sh * sin(phi), ch, hh);
            double c = dot3(wo, hh);
            for (int a = 0; a < 3; ++a) wi[a] = 2.0 * c * hh[a] - wo[a];
        }
        double f[3], pdf;
        vertex_brdf_h(R, h.id, n, wo, wi, glossy ? hh : NULL, f, &pdf, &Pd, amb);
        if (pdf <= 0.0) return;
        for (int c = 0; c < 3; ++c) beta[c] *= f[c] / pdf;
        for (int a = 0; a < 3; ++a) { o[a] = xo[a]; d[a] = wi[a]; }
        skip = h.id;
        pdf_prev = pdf;
    }
}

/* ------------------------------------------------------------------ */
/* Ranges of refinement samples over the decisions float32 can flip     */
/* ------------------------------------------------------------------ */
/* A float32 path may take the other side of any decision that lies
 * within its rounding of a threshold, and along a path that rounding
 * grows: the hit point of a ray whose origin is uncertain by e_o and whose
 * direction by e_d is uncertain by (e_o + t e_d) / |cos| on the surface it
 * meets, a glossy reflection keeps its incoming direction's uncertainty,
 * and every float32 step adds a few units of 2^-24.  For each sample the
 * functions below carry (e_o, e_d) along every branch and follow every
 * alternative within them:
 *   - every hit a perturbed ray may report (closest() with its window
 *     widened to the ray's uncertainty), both facings where grazing, a miss
 *     where one is possible;
 *   - both emitter triangles where the area-sampling uniform lies within
 *     1e-6 A of a cumulative boundary;
 *   - zero for an emitter sample whose cosine at the emitter or at the
 *     receiver is within its uncertainty (at least 1e-5) of 0; lit and
 *     unlit where the shadow ray's candidates disagree about reaching the
 *     sampled triangle;
 *   - the specular lobe on and off where n.wo is within max(1e-6, 2 e_d)
 *     of 1e-2; with and without the specular part where wo.h is within
 *     max(1e-5, ...) of 0; with and without the n.wi > 0 branch where n.wi
 *     is within max(1e-5, ...) of 0;
 *   - both lobes where the lobe uniform lies within 1e-5 of P_d;
 *   - both tangent frames where the normal's z is within 2e-7 of the
 *     frame branch;
 *   - GGX D at a recomputed half vector tilted by -tau, 0, +tau, tau =
 *     max(2e-6 rad, the directions' uncertainty), where D changes by more
 *     than 1e-4 under that tilt;
 *   - every voxel the hit point may fall in.
 * Each combination of alternatives accumulates its terms in the nominal
 * order, so without any alternative the range is the nominal value
 * exactly.  Every term is non-negative; a sample whose hit points become
 * uncertain by more than 1e-4 of the scene size, whose alternatives need
 * more than OR_RANGE_BUDGET path segments, or whose ray meets more
 * candidates than closest() holds, gets the range [0, inf]. */
#define OR_RANGE_BUDGET 4096
#define OR_TILT 2e-6
#define OR_U32 (1.0 / 16777216.0)     /* 2^-24 */

typedef struct { int32_t id; double t; int front; } oalt;
#define OMAXALT (2 * OMAXC + 4)

typedef struct {
    const refine_job* R;
    uint32_t pid, s, lobe;
    int segments;
    int unbounded;
    double mag;                  /* largest |coordinate| of the scene box */
    double Lmin[3], Lmax[3];
} rwalk;

static void rw_leaf(rwalk* W, const double L[3])
{
    for (int c = 0; c < 3; ++c) {
        if (L[c] < W->Lmin[c]) W->Lmin[c] = L[c];
        if (L[c] > W->Lmax[c]) W->Lmax[c] = L[c];
    }
}

static void alt_add(oalt* a, int* n, int32_t id, double t, int front)
{
    for (int i = 0; i < *n; ++i) if (a[i].id == id && (id < 0 || a[i].front == front)) return;
    if (*n < OMAXALT) { a[*n].id = id; a[*n].t = t; a[*n].front = front; ++*n; }
}

/* Every hit a float32 ray o + t d may report (skip excluded), for an
 * origin uncertain by eo and a direction uncertain by ed. */
static int hit_alts(const refine_job* R, const double o[3], const double d[3], int skip,
                    double eo, double ed, oalt* a, int* unbounded)
{
    double eta = R->eta;
    if (2.0 * eo / R->S->L > eta) eta = 2.0 * eo / R->S->L;
    if (2.0 * ed > eta) eta = 2.0 * ed;
    ocands c;
    closest(R->S, o, d, skip, eta, &c);
    int n = 0;
    if (c.overflow) *unbounded = 1;
    alt_add(a, &n, c.nominal.id, c.nominal.t, c.nominal.front);
    if (c.nominal.id >= 0 && c.nominal.front_amb) alt_add(a, &n, c.nominal.id, c.nominal.t, !c.nominal.front);
    for (int i = 0; i < c.n; ++i) {
        alt_add(a, &n, c.c[i].id, c.c[i].t, c.c[i].front);
        if (c.c[i].front_amb) alt_add(a, &n, c.c[i].id, c.c[i].t, !c.c[i].front);
    }
    if (c.miss_possible) alt_add(a, &n, -1, INFINITY, 0);
    return n;
}

/* Emitter triangles (indices into R->emit) that a float32 search of the
 * cumulative areas may pick for uniform u0; returns how many (1 to 3). */
static int emitter_alts(const refine_job* R, double u0, int* k)
{
    double target = u0 * R->A;
    int lo = 0, hi = R->n_emit - 1;
    while (lo < hi) {
        int mid = (lo + hi) / 2;
        if (R->cdf[mid] > target) hi = mid; else lo = mid + 1;
    }
    int n = 0;
    k[n++] = lo;
    if (R->n_emit > 1) {
        if (fabs(R->cdf[lo] - target) < 1e-6 * R->A && lo + 1 < R->n_emit) k[n++] = lo + 1;
        if (lo > 0 && fabs(R->cdf[lo - 1] - target) < 1e-6 * R->A) k[n++] = lo - 1;
    }
    return n;
}

/* The point the area sample draws on emitter list entry k. */
static int emitter_point(const refine_job* R, int k, const double u[4], double y[3])
{
    const otri* tr = &R->S->tri[R->emit[k]];
    double r1 = sqrt(u[1]);
    double b0 = 1.0 - r1, b1 = r1 * (1.0 - u[2]), b2 = r1 * u[2];
    for (int a = 0; a < 3; ++a) y[a] = b0 * tr->v0[a] + b1 * tr->v1[a] + b2 * tr->v2[a];
    return R->emit[k];
}

/* Frame of onb() with its branch forced (s = +1 or -1). */
static void onb_forced(const double n[3], double s, double t[3], double b[3])
{
    double a = -1.0 / (s + n[2]);
    double c = n[0] * n[1] * a;
    t[0] = 1.0 + s * n[0] * n[0] * a; t[1] = s * c; t[2] = -s * n[0];
    b[0] = c; b[1] = s + n[1] * n[1] * a; b[2] = -n[1];
}

/* GGX D at polar angle theta of the half vector. */
static double ggx_D_theta(double th, double a2)
{
    double sn = sin(th), cs = cos(th);
    double den = sn * sn + a2 * cs * cs;
    return a2 / (OPI * den * den);
}

typedef struct { double f[3]; double pdf; } bvar;
#define OMAXBV 16

/* The values (f, pdf) that vertex_brdf_h may take for a float32 evaluation,
 * with the specular lobe forced on or off (spec), wo uncertain by ed_o and
 * wi by ed_i.  The first entry is the nominal one, computed as
 * vertex_brdf_h computes it. */
static int brdf_alts(const refine_job* R, int t, const double n[3], const double wo[3],
                     const double wi[3], const double* hs, int spec, double ed_o, double ed_i,
                     bvar* out)
{
    const double a[3] = {R->ma[3*t], R->ma[3*t+1], R->ma[3*t+2]};
    const double sg = R->ms[t], m = R->mm[t];
    const double al = sg * sg, a2 = al * al;
    double kd[3], ks[3], kdm = 0, ksm = 0;
    for (int c = 0; c < 3; ++c) {
        kd[c] = a[c] * (1.0 - m); ks[c] = 0.04 * (1.0 - m) + a[c] * m;
        kdm += R->ma[3*t+c] * (1.0 - m); ksm += 0.04 * (1.0 - m) + R->ma[3*t+c] * m;
    }
    double Pd = kdm / (kdm + ksm);
    if (Pd < 0.1) Pd = 0.1;
    if (Pd > 0.9) Pd = 0.9;
    if (!spec) Pd = 1.0;
    const double mu_o = dot3(n, wo), mu_i0 = dot3(n, wi);
    const double w_mu = fmax(1e-5, 2.0 * ed_i), w_co = fmax(1e-5, 2.0 * (ed_o + ed_i));
    const double tilt = fmax(OR_TILT, ed_o + ed_i);
    int nv = 0;
    /* n.wi branch: nominal first, the other side where within its window of 0 */
    const int mu_cases[2] = {mu_i0 > 0.0, !(mu_i0 > 0.0)};
    const int n_mu = fabs(mu_i0) < w_mu ? 2 : 1;
    for (int im = 0; im < n_mu; ++im) {
        if (!mu_cases[im]) {
            bvar z = {{0, 0, 0}, 0.0};
            if (nv < OMAXBV) out[nv++] = z;
            continue;
        }
        const double mu_i = mu_i0 > 0.0 ? mu_i0 : (mu_i0 < 0.0 ? -mu_i0 : 1e-300);
        bvar base;
        for (int c = 0; c < 3; ++c) base.f[c] = kd[c] * mu_i / OPI;
        base.pdf = Pd * mu_i / OPI;
        if (!spec) { if (nv < OMAXBV) out[nv++] = base; continue; }
        double h[3] = {wi[0] + wo[0], wi[1] + wo[1], wi[2] + wo[2]};
        if (hs) { h[0] = hs[0]; h[1] = hs[1]; h[2] = hs[2]; }
        normalize3(h);
        const double ch = dot3(n, h), co0 = dot3(wo, h);
        /* wo.h branch */
        const int co_cases[2] = {ch > 0.0 && co0 > 0.0, !(ch > 0.0 && co0 > 0.0)};
        const int n_co = (fabs(co0) < w_co && ch > 0.0) ? 2 : 1;
        for (int ic = 0; ic < n_co; ++ic) {
            if (!co_cases[ic]) { if (nv < OMAXBV) out[nv++] = base; continue; }
            const double co = co0 > 0.0 ? co0 : (co0 < 0.0 ? -co0 : 1e-300);
            double Ds[3];
            int nD = 1;
            Ds[0] = ggx_D(ch, a2);
            if (!hs) {
                double cr[3];
                cross3(n, h, cr);
                if (ggx_log_slope(ch, norm3(cr), a2) * tilt > 1e-4) {
                    double th = atan2(norm3(cr), ch);
                    Ds[nD++] = ggx_D_theta(th > tilt ? th - tilt : 0.0, a2);
                    Ds[nD++] = ggx_D_theta(th + tilt, a2);
                }
            }
            const double G = smith_g1(mu_i, a2) * smith_g1(mu_o, a2);
            const double F1 = pow(1.0 - co, 5.0), F0 = 1.0 - F1;
            for (int iD = 0; iD < nD && nv < OMAXBV; ++iD) {
                bvar v = base;
                const double D = Ds[iD];
                for (int c = 0; c < 3; ++c) v.f[c] += (ks[c] * F0 + F1) * D * G / (4.0 * mu_o);
                v.pdf += (1.0 - Pd) * D * ch / (4.0 * co);
                out[nv++] = v;
            }
        }
    }
    return nv;
}

static void path_range(rwalk* W, const double o[3], const double d[3], int skip, double pdf_prev,
                       const double beta[3], int depth, const double L[3], double eo, double ed);

/* A path vertex on alternative hit h of the ray (o, d) at path depth
 * `depth`, with L accumulated so far and the hit point uncertain by ex, the
 * incoming direction by ed: next-event estimation, then every
 * continuation. */
static void vertex_range(rwalk* W, const double o[3], const double d[3], const oalt* h,
                         const double beta[3], int depth, const double L[3], int nominal_facing,
                         double ex, double ed)
{
    const refine_job* R = W->R;
    const oscene* S = R->S;
    const otri* tr = &S->tri[h->id];
    double x[3], n[3] = {tr->ng[0], tr->ng[1], tr->ng[2]}, wo[3] = {-d[0], -d[1], -d[2]};
    normalize3(n);
    for (int a = 0; a < 3; ++a) x[a] = o[a] + h->t * d[a];
    int flip = dot3(n, wo) < 0;
    if (!nominal_facing) flip = !flip;
    if (flip) for (int a = 0; a < 3; ++a) n[a] = -n[a];
    const int famb = fabs(n[2] - OR_ONB_BRANCH) < 2e-7;
    double xo[3];
    for (int a = 0; a < 3; ++a) xo[a] = x[a] + S->eps * n[a];
    const double exo = ex + 4.0 * OR_U32 * W->mag;     /* the offset origin in float32 */
    const uint32_t lane = W->lobe | ((uint32_t)depth << 9);
    const double mu_o = dot3(n, wo);
    const int spec_nom = mu_o > 1e-2;
    const int n_spec = fabs(mu_o - 1e-2) < fmax(1e-6, 2.0 * ed) ? 2 : 1;
    for (int isp = 0; isp < n_spec; ++isp) {
        const int spec = isp == 0 ? spec_nom : !spec_nom;
        /* next-event estimation: every accumulated value it may leave */
        double Ln[64][3];
        int nn = 0;
        if (R->mis && R->n_emit > 0) {
            double u[4];
            philox_words(W->pid, W->s, lane | 0x100u, R->request_id, R->seed, u);
            int ks[3];
            const int nk = emitter_alts(R, u[0], ks);
            for (int ik = 0; ik < nk; ++ik) {
                double y[3], wl[3];
                const int e = emitter_point(R, ks[ik], u, y);
                sub3(y, xo, wl);
                double dist = norm3(wl);
                for (int a = 0; a < 3; ++a) wl[a] /= dist;
                const double ed_sh = exo / dist + 4.0 * OR_U32;
                const otri* te = &S->tri[e];
                double ce = -dot3(wl, te->ng) / te->area2;
                int zero = !(ce > 0) || fabs(ce) < fmax(1e-5, 2.0 * ed_sh);
                if (zero && nn < 64) { for (int c = 0; c < 3; ++c) Ln[nn][c] = L[c]; ++nn; }
                if (!(ce > 0)) continue;
                bvar bv[OMAXBV];
                const int nb = brdf_alts(R, h->id, n, wo, wl, NULL, spec, ed, ed_sh, bv);
                oalt sa[OMAXALT];
                int sna = -1;
                for (int ib = 0; ib < nb; ++ib) {
                    const double* f = bv[ib].f;
                    const double pb = bv[ib].pdf;
                    if (!(f[0] > 0 || f[1] > 0 || f[2] > 0)) {
                        if (nn < 64) { for (int c = 0; c < 3; ++c) Ln[nn][c] = L[c]; ++nn; }
                        continue;
                    }
                    if (sna < 0) sna = hit_alts(R, xo, wl, h->id, exo, ed_sh, sa, &W->unbounded);
                    int lit = 0, unlit = 0;
                    for (int i = 0; i < sna; ++i) { if (sa[i].id == e) lit = 1; else unlit = 1; }
                    if (unlit && nn < 64) { for (int c = 0; c < 3; ++c) Ln[nn][c] = L[c]; ++nn; }
                    if (lit && nn < 64) {
                        double pl = dist * dist / (R->A * ce);
                        double w = pl * pl / (pl * pl + pb * pb);
                        for (int c = 0; c < 3; ++c) Ln[nn][c] = L[c] + beta[c] * w * S->Le[3*e+c] * f[c] / pl;
                        ++nn;
                    }
                }
            }
            if (nn >= 64) W->unbounded = 1;
        } else {
            for (int c = 0; c < 3; ++c) Ln[0][c] = L[c];
            nn = 1;
        }
        /* BRDF sample: every lobe, frame and evaluation alternative */
        double u[4];
        philox_words(W->pid, W->s, lane, R->request_id, R->seed, u);
        double kdm = 0, ksm = 0;
        const double mm = R->mm[h->id];
        for (int c = 0; c < 3; ++c) {
            kdm += R->ma[3*h->id+c] * (1.0 - mm);
            ksm += 0.04 * (1.0 - mm) + R->ma[3*h->id+c] * mm;
        }
        double Pd = kdm / (kdm + ksm);
        if (Pd < 0.1) Pd = 0.1;
        if (Pd > 0.9) Pd = 0.9;
        if (!spec) Pd = 1.0;
        const int glossy_nom = !(u[2] < Pd);
        const int n_lobe = fabs(u[2] - Pd) < 1e-5 ? 2 : 1;
        const double s_nom = n[2] >= OR_ONB_BRANCH ? 1.0 : -1.0;
        const int n_frame = famb ? 2 : 1;
        for (int in_ = 0; in_ < nn; ++in_) {
            for (int il = 0; il < n_lobe; ++il) {
                const int glossy = il == 0 ? glossy_nom : !glossy_nom;
                /* a reflection keeps the incoming direction's uncertainty */
                const double ed_i = (glossy ? ed : 0.0) + 8.0 * OR_U32;
                for (int iff = 0; iff < n_frame; ++iff) {
                    double tb[3], bb[3], wi[3], hh[3];
                    if (iff == 0) onb(n, tb, bb); else onb_forced(n, -s_nom, tb, bb);
                    if (!glossy) {
                        double rad = sqrt(u[0]), phi = 2.0 * OPI * u[1];
                        to_world(tb, bb, n, rad * cos(phi), rad * sin(phi), sqrt(1.0 - u[0]), wi);
                    } else {
                        const double al = (double)R->ms[h->id] * (double)R->ms[h->id], a2 = al * al;
                        double cos2 = (1.0 - u[0]) / (1.0 + (a2 - 1.0) * u[0]);
                        double ch = sqrt(cos2), sh = sqrt(fmax(0.0, 1.0 - cos2)), phi = 2.0 * OPI * u[1];
                        to_world(tb, bb, n, sh * cos(phi), sh * sin(phi), ch, hh);
                        double c = dot3(wo, hh);
                        for (int a = 0; a < 3; ++a) wi[a] = 2.0 * c * hh[a] - wo[a];
                    }
                    bvar bv[OMAXBV];
                    const int nb = brdf_alts(R, h->id, n, wo, wi, glossy ? hh : NULL, spec, ed, ed_i, bv);
                    for (int ib = 0; ib < nb; ++ib) {
                        if (bv[ib].pdf <= 0.0) { rw_leaf(W, Ln[in_]); continue; }
                        double b2[3];
                        for (int c = 0; c < 3; ++c) b2[c] = beta[c] * (bv[ib].f[c] / bv[ib].pdf);
                        path_range(W, xo, wi, h->id, bv[ib].pdf, b2, depth + 1, Ln[in_], exo, ed_i);
                        if (W->unbounded) return;
                    }
                }
            }
        }
    }
}

/* Every value the path radiance may take from the ray (o, d) on (see the
 * header of this section), each branch adding to L in the nominal order;
 * beta and pdf_prev as in path_radiance; eo, ed the uncertainty of the
 * ray's origin and direction. */
static void path_range(rwalk* W, const double o[3], const double d[3], int skip, double pdf_prev,
                       const double beta[3], int depth, const double L[3], double eo, double ed)
{
    const refine_job* R = W->R;
    const oscene* S = R->S;
    if (W->unbounded) return;
    if (++W->segments > OR_RANGE_BUDGET) { W->unbounded = 1; return; }
    oalt al[OMAXALT];
    const int na = hit_alts(R, o, d, skip, eo, ed, al, &W->unbounded);
    if (W->unbounded) return;
    const double dl = norm3(d);
    for (int i = 0; i < na; ++i) {
        const oalt* h = &al[i];
        double Lt[3] = {L[0], L[1], L[2]};
        if (h->id < 0) {
            double Le[3];
            env_lookup(S, d, Le);
            for (int c = 0; c < 3; ++c) Lt[c] += beta[c] * Le[c];
            rw_leaf(W, Lt);
            continue;
        }
        /* the hit point's uncertainty on the surface */
        const otri* tr = &S->tri[h->id];
        const double cs = fabs(dot3(d, tr->ng)) / (dl * tr->area2);
        const double ex = (eo + h->t * ed) / fmax(cs, 1e-3) + 4.0 * OR_U32 * (W->mag + h->t);
        if (is_emitter(S, h->id)) {
            if (h->front) {
                double w = 1.0;
                if (R->mis && R->n_emit > 0) {
                    double ce = fabs(dot3(d, tr->ng)) / tr->area2;
                    double pl = h->t * h->t / (R->A * ce);
                    w = pdf_prev * pdf_prev / (pdf_prev * pdf_prev + pl * pl);
                }
                for (int c = 0; c < 3; ++c) Lt[c] += beta[c] * w * S->Le[3*h->id+c];
            }
            rw_leaf(W, Lt);
            continue;
        }
        if ((double)R->ms[h->id] > R->sigma_c) {
            double p[3] = {o[0] + h->t * d[0], o[1] + h->t * d[1], o[2] + h->t * d[2]};
            if (S->vox) {
                double ext = 0.0;
                for (int a = 0; a < 3; ++a) ext = fmax(ext, S->shi[a] - S->slo[a]);
                double vl[3], vh[3], A[3], B[3];
                voxel_range_w(S, p, fmax(1e-3, 2.0 * ex * S->vox_r / ext), vl, vh);
                for (int c = 0; c < 3; ++c) { A[c] = Lt[c] + beta[c] * vl[c]; B[c] = Lt[c] + beta[c] * vh[c]; }
                rw_leaf(W, A);
                rw_leaf(W, B);
            } else {
                double C[3];
                cache_at(S, h->id, p, C);
                for (int c = 0; c < 3; ++c) Lt[c] += beta[c] * C[c];
                rw_leaf(W, Lt);
            }
            continue;
        }
        if (depth > R->max_depth) { rw_leaf(W, Lt); continue; }
        if (ex > 1e-4 * S->L) { W->unbounded = 1; return; }
        /* the facing FP64 gives this triangle, or the other one (grazing) */
        const int nominal_facing = h->front == (dot3(d, tr->ng) < 0.0);
        vertex_range(W, o, d, h, beta, depth, Lt, nominal_facing, ex, ed);
        if (W->unbounded) return;
    }
}

/* Range of one sample's six values (see the section header): the
 * emitter sample at the query point, then the lobe sample's path; lo / hi
 * receive the extremes, or [0, inf] when unbounded (returns 1 then). */
static int sample_range(const refine_job* R, const double o[3], const double n[3], const double wo[3],
                        const double tb[3], const double bb[3], int32_t skip, uint32_t pid,
                        uint32_t s, uint32_t lobe, double a2, double g1o, double mu_o,
                        double lo[6], double hi[6])
{
    const oscene* S = R->S;
    rwalk W;
    memset(&W, 0, sizeof(W));
    W.R = R; W.pid = pid; W.s = s; W.lobe = lobe;
    for (int a = 0; a < 3; ++a) W.mag = fmax(W.mag, fmax(fabs(S->slo[a]), fabs(S->shi[a])));
    const double eo = 4.0 * OR_U32 * W.mag, ed = 8.0 * OR_U32;
    /* every six-value partial sum the emitter sample at x may leave */
    double N6[64][6];
    int nn = 0;
    if (R->mis && R->n_emit > 0) {
        double u[4];
        philox_words(pid, s, lobe | 0x100u, R->request_id, R->seed, u);
        int ks[3];
        const int nk = emitter_alts(R, u[0], ks);
        for (int ik = 0; ik < nk; ++ik) {
            double y[3], wl[3];
            const int e = emitter_point(R, ks[ik], u, y);
            sub3(y, o, wl);
            double dist = norm3(wl);
            for (int a = 0; a < 3; ++a) wl[a] /= dist;
            const double ed_sh = eo / dist + 4.0 * OR_U32;
            const double wz = fmax(1e-5, 2.0 * ed_sh);
            const otri* te = &S->tri[e];
            double ce = -dot3(wl, te->ng) / te->area2;
            double mu_i = dot3(n, wl);
            /* the zero contribution, wherever a decision may zero it */
            const int maybe_zero = !(ce > 0 && mu_i > 0) || fabs(ce) < wz || fabs(mu_i) < wz;
            if (maybe_zero && nn < 64) { memset(N6[nn], 0, sizeof(N6[nn])); ++nn; }
            const double mu_e = mu_i > 0 ? mu_i : (mu_i < 0 ? -mu_i : 1e-300);
            if (!(ce > 0) || !(mu_i > 0 || fabs(mu_i) < wz)) continue;
            double g0s[3], g1s[3], pbs[3];
            int ng = 0;
            if (lobe == 0) { g0s[0] = mu_e / OPI; g1s[0] = 0; pbs[0] = mu_e / OPI; ng = 1; }
            else {
                double h[3] = {wl[0] + wo[0], wl[1] + wo[1], wl[2] + wo[2]};
                normalize3(h);
                double ch = dot3(n, h), c = dot3(wo, h);
                const int c_ok = ch > 0 && c > 0, c_near = fabs(c) < wz && ch > 0;
                if ((!c_ok || c_near) && nn < 64) { memset(N6[nn], 0, sizeof(N6[nn])); ++nn; }
                if (!c_ok && !c_near) continue;
                const double cc = c > 0 ? c : (c < 0 ? -c : 1e-300);
                const double tilt = fmax(OR_TILT, ed + ed_sh);
                double cr[3];
                cross3(n, h, cr);
                double Ds[3];
                int nD = 1;
                Ds[0] = ggx_D(ch, a2);
                if (ggx_log_slope(ch, norm3(cr), a2) * tilt > 1e-4) {
                    double th = atan2(norm3(cr), ch);
                    Ds[nD++] = ggx_D_theta(th > tilt ? th - tilt : 0.0, a2);
                    Ds[nD++] = ggx_D_theta(th + tilt, a2);
                }
                for (int iD = 0; iD < nD; ++iD) {
                    double D = Ds[iD], G = smith_g1(mu_e, a2) * g1o;
                    double F1 = pow(1.0 - cc, 5.0);
                    g0s[ng] = (1.0 - F1) * D * G / (4.0 * mu_o);
                    g1s[ng] = F1 * D * G / (4.0 * mu_o);
                    pbs[ng] = D * ch / (4.0 * cc);
                    ++ng;
                }
            }
            oalt sa[OMAXALT];
            int sna = -1;
            for (int ig = 0; ig < ng; ++ig) {
                if (!(g0s[ig] > 0 || g1s[ig] > 0)) {
                    if (nn < 64) { memset(N6[nn], 0, sizeof(N6[nn])); ++nn; }
                    continue;
                }
                if (sna < 0) sna = hit_alts(R, o, wl, skip, eo, ed_sh, sa, &W.unbounded);
                int lit = 0, unlit = 0;
                for (int i = 0; i < sna; ++i) { if (sa[i].id == e) lit = 1; else unlit = 1; }
                if (unlit && nn < 64) { memset(N6[nn], 0, sizeof(N6[nn])); ++nn; }
                if (lit && nn < 64) {
                    double pl = dist * dist / (R->A * ce);
                    double w = pl * pl / (pl * pl + pbs[ig] * pbs[ig]);
                    for (int c = 0; c < 3; ++c) {
                        N6[nn][c] = 0.0 + w * S->Le[3*e+c] * g0s[ig] / pl;
                        N6[nn][3+c] = 0.0 + w * S->Le[3*e+c] * g1s[ig] / pl;
                    }
                    ++nn;
                }
            }
        }
        if (nn >= 64) W.unbounded = 1;
    } else {
        memset(N6[0], 0, sizeof(N6[0]));
        nn = 1;
    }
    /* the lobe sample at x, as in the bake */
    double u[4];
    philox_words(pid, s, lobe, R->request_id, R->seed, u);
    strat_uv(s, lobe == 0 ? R->spp_d : R->spp_s, &u[0], &u[1]);
    double wi[3], W0 = 1.0, W1 = 0.0, pb = 0.0;
    int can_zero = 0, can_go = 1;
    if (lobe == 0) {
        double rad = sqrt(u[0]), phi = 2.0 * OPI * u[1];
        to_world(tb, bb, n, rad * cos(phi), rad * sin(phi), sqrt(1.0 - u[0]), wi);
        pb = sqrt(1.0 - u[0]) / OPI;
    } else {
        double cos2 = (1.0 - u[0]) / (1.0 + (a2 - 1.0) * u[0]);
        double ch = sqrt(cos2), sh = sqrt(fmax(0.0, 1.0 - cos2)), phi = 2.0 * OPI * u[1];
        double h[3];
        to_world(tb, bb, n, sh * cos(phi), sh * sin(phi), ch, h);
        double c = dot3(wo, h);
        for (int a = 0; a < 3; ++a) wi[a] = 2.0 * c * h[a] - wo[a];
        double mu_i = dot3(n, wi);
        const int valid = mu_i > 0.0 && c > 0.0;
        const int near = fabs(mu_i) < 1e-5 || fabs(c) < 1e-5;
        can_zero = !valid || near;
        can_go = valid || near;
        const double mu_e = mu_i > 0 ? mu_i : (mu_i < 0 ? -mu_i : 1e-300);
        const double cc = c > 0 ? c : (c < 0 ? -c : 1e-300);
        double G = smith_g1(mu_e, a2) * g1o, w = G * cc / (mu_o * ch);
        double F1 = pow(1.0 - cc, 5.0);
        W0 = (1.0 - F1) * w;
        W1 = F1 * w;
        pb = ggx_D(ch, a2) * ch / (4.0 * cc);
    }
    double Lmin[3] = {0, 0, 0}, Lmax[3] = {0, 0, 0};
    if (can_go) {
        for (int c = 0; c < 3; ++c) { W.Lmin[c] = INFINITY; W.Lmax[c] = -INFINITY; }
        const double one[3] = {1, 1, 1}, zero3[3] = {0, 0, 0};
        path_range(&W, o, wi, skip, pb, one, 1, zero3, eo, ed);
        for (int c = 0; c < 3; ++c) { Lmin[c] = W.Lmin[c]; Lmax[c] = W.Lmax[c]; }
    }
    if (W.unbounded) {
        for (int i = 0; i < 6; ++i) { lo[i] = 0.0; hi[i] = INFINITY; }
        return 1;
    }
    for (int i = 0; i < 6; ++i) { lo[i] = INFINITY; hi[i] = -INFINITY; }
    for (int k = 0; k < nn; ++k) {
        for (int c = 0; c < 3; ++c) {
            double v0[3], v1[3];
            int m = 0;
            if (can_go) {
                v0[m] = N6[k][c] + W0 * Lmin[c]; v1[m] = N6[k][3+c] + W1 * Lmin[c]; ++m;
                v0[m] = N6[k][c] + W0 * Lmax[c]; v1[m] = N6[k][3+c] + W1 * Lmax[c]; ++m;
            }
            if (can_zero) { v0[m] = N6[k][c]; v1[m] = N6[k][3+c]; ++m; }
            for (int j = 0; j < m; ++j) {
                lo[c] = fmin(lo[c], v0[j]);   hi[c] = fmax(hi[c], v0[j]);
                lo[3+c] = fmin(lo[3+c], v1[j]); hi[3+c] = fmax(hi[3+c], v1[j]);
            }
        }
    }
    return 0;
}

static void refine_point(refine_job* R, int64_t p)
{
    const oscene* S = R->S;
    const int K = R->K, W = 3 + 6 * K;
    double* out = R->out + (size_t)W * p;
    for (int i = 0; i < W; ++i) out[i] = 0.0;
    double x[3], n[3], wo[3];
    for (int a = 0; a < 3; ++a) { x[a] = R->qx[3*p+a]; n[a] = R->qn[3*p+a]; wo[a] = R->qwo[3*p+a]; }
    normalize3(n);
    normalize3(wo);
    const int32_t skip = R->qtri[p];
    double o[3];
    for (int a = 0; a < 3; ++a) o[a] = x[a] + S->eps * n[a];
    double tb[3], bb[3];
    onb(n, tb, bb);
    const double mu_o = dot3(n, wo);
    const uint32_t pid = R->point_base + (uint32_t)p;
    for (int lobe = 0; lobe <= K; ++lobe) {
        const int Sn = lobe == 0 ? R->spp_d : R->spp_s;
        if (lobe > 0 && mu_o <= 1e-2) continue;
        double a2 = 0, g1o = 0;
        if (lobe > 0) {
            const double al = R->sigma[lobe - 1] * R->sigma[lobe - 1];
            a2 = al * al;
            g1o = smith_g1(mu_o, a2);
        }
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int s = 0; s < Sn; ++s) {
            int amb = 0;
            double c6[6] = {0, 0, 0, 0, 0, 0};
            /* emitter sample at x (MIS) */
            if (R->mis && R->n_emit > 0) {
                double u[4], y[3], wl[3];
                philox_words(pid, (uint32_t)s, (uint32_t)lobe | 0x100u, R->request_id, R->seed, u);
                int e = emitter_sample(R, u, y, &amb);
                sub3(y, o, wl);
                double dist = norm3(wl);
                for (int a = 0; a < 3; ++a) wl[a] /= dist;
                const otri* te = &S->tri[e];
                double ce = -dot3(wl, te->ng) / te->area2;
                double mu_i = dot3(n, wl);
                if (fabs(ce) < 1e-5 || fabs(mu_i) < 1e-5) amb = 1;
                double g0 = 0, g1 = 0, pb = 0;
                if (ce > 0 && mu_i > 0) {
                    if (lobe == 0) { g0 = mu_i / OPI; pb = mu_i / OPI; }
                    else {
                        double h[3] = {wl[0] + wo[0], wl[1] + wo[1], wl[2] + wo[2]};
                        normalize3(h);
                        double ch = dot3(n, h), c = dot3(wo, h);
                        if (fabs(c) < 1e-5) amb = 1;
                        double cr[3];
                        cross3(n, h, cr);
                        if (ggx_log_slope(ch, norm3(cr), a2) > OR_SLOPE_LIMIT) amb = 1;
                        if (ch > 0 && c > 0) {
                            double D = ggx_D(ch, a2), G = smith_g1(mu_i, a2) * g1o;
                            double F1 = pow(1.0 - c, 5.0);
                            g0 = (1.0 - F1) * D * G / (4.0 * mu_o);
                            g1 = F1 * D * G / (4.0 * mu_o);
                            pb = D * ch / (4.0 * c);
                        }
                    }
                }
                if (g0 > 0 || g1 > 0) {
                    ohit vh;
                    trace_flag(R, o, wl, skip, &vh, &amb);
                    if (vh.id == e) {
                        double pl = dist * dist / (R->A * ce);
                        double w = pl * pl / (pl * pl + pb * pb);
                        for (int c = 0; c < 3; ++c) {
                            c6[c] += w * S->Le[3*e+c] * g0 / pl;
                            c6[3+c] += w * S->Le[3*e+c] * g1 / pl;
                        }
                    }
                }
            }
            /* lobe sample at x, as in the bake */
            double u[4];
            philox_words(pid, (uint32_t)s, (uint32_t)lobe, R->request_id, R->seed, u);
            strat_uv((uint32_t)s, Sn, &u[0], &u[1]);
            double wi[3], W0 = 1.0, W1 = 0.0, pb = 0.0;
            int valid = 1;
            if (lobe == 0) {
                double rad = sqrt(u[0]), phi = 2.0 * OPI * u[1];
                to_world(tb, bb, n, rad * cos(phi), rad * sin(phi), sqrt(1.0 - u[0]), wi);
                pb = sqrt(1.0 - u[0]) / OPI;
            } else {
                double cos2 = (1.0 - u[0]) / (1.0 + (a2 - 1.0) * u[0]);
                double ch = sqrt(cos2), sh = sqrt(fmax(0.0, 1.0 - cos2)), phi = 2.0 * OPI * u[1];
                double h[3];
                to_world(tb, bb, n, sh * cos(phi), sh * sin(phi), ch, h);
                double c = dot3(wo, h);
                for (int a = 0; a < 3; ++a) wi[a] = 2.0 * c * h[a] - wo[a];
                double mu_i = dot3(n, wi);
                if (fabs(mu_i) < 1e-5 || fabs(c) < 1e-5) amb = 1;
                if (mu_i <= 0.0 || c <= 0.0) valid = 0;
                else {
                    double G = smith_g1(mu_i, a2) * g1o, w = G * c / (mu_o * ch);
                    double F1 = pow(1.0 - c, 5.0);
                    W0 = (1.0 - F1) * w;
                    W1 = F1 * w;
                    pb = ggx_D(ch, a2) * ch / (4.0 * c);
                }
            }
            if (valid) {
                double L[3];
                path_radiance(R, o, wi, skip, pb, pid, (uint32_t)s, (uint32_t)lobe, L, &amb);
                for (int c = 0; c < 3; ++c) { c6[c] += W0 * L[c]; c6[3+c] += W1 * L[c]; }
            }
            for (int i = 0; i < 6; ++i) acc[i] += c6[i];
            if (R->per_sample) {
                double* ps = R->per_sample + ((size_t)(p * (K + 1) + lobe) * R->smax + s) * 6;
                for (int i = 0; i < 6; ++i) ps[i] = c6[i];
            }
            if (R->amb) R->amb[(size_t)(p * (K + 1) + lobe) * R->smax + s] = (uint8_t)amb;
            if (R->ps_lo) {
                const size_t at = (size_t)(p * (K + 1) + lobe) * R->smax + s;
                int unb = sample_range(R, o, n, wo, tb, bb, skip, pid, (uint32_t)s, (uint32_t)lobe,
                                       a2, g1o, mu_o, R->ps_lo + 6 * at, R->ps_hi + 6 * at);
                if (lobe == 0) for (int c = 3; c < 6; ++c) { R->ps_lo[6*at+c] = 0.0; R->ps_hi[6*at+c] = 0.0; }
                if (R->unb) R->unb[at] = (uint8_t)unb;
            }
        }
        if (lobe == 0) for (int c = 0; c < 3; ++c) out[c] = acc[c] / Sn;
        else for (int c = 0; c < 3; ++c) {
            out[3 + 3*(lobe-1) + c] = acc[c] / Sn;
            out[3 + 3*K + 3*(lobe-1) + c] = acc[3+c] / Sn;
        }
    }
}

static void* refine_worker(void* arg)
{
    refine_job* R = (refine_job*)arg;
    for (;;) {
        int64_t p = __atomic_fetch_add(&R->next, 1, __ATOMIC_RELAXED);
        if (p >= R->N) break;
        refine_point(R, p);
    }
    return NULL;
}

/* Stage-3 bake.  mat_a [T,3], mat_sigma [T], mat_m [T] per triangle.
 * Outputs as oracle_bake (nominal only); per_sample (nullable) gets every
 * sample's 6 values (L_d uses the first 3), amb (nullable) 1 for samples
 * whose path takes a decision within rounding of a threshold.  With
 * per_sample and eta > 0, ps_lo / ps_hi (nullable) receive each sample's
 * range over those decisions (sample_range) and unb (nullable) 1 where the
 * range is [0, inf]. */
int oracle_refine(const oscene* S, const float* mat_a, const float* mat_sigma, const float* mat_m,
                  const float* qx, const float* qn, const float* qwo, const int32_t* qtri, int64_t N,
                  uint64_t seed, uint32_t request_id, uint32_t point_base, int spp_d, int spp_s,
                  int K, const double* sigma, double sigma_c, int max_depth, int mis, double eta,
                  int nthreads, double* out, double* per_sample, uint8_t* amb,
                  double* ps_lo, double* ps_hi, uint8_t* unb)
{
    refine_job R;
    memset(&R, 0, sizeof(R));
    R.S = S; R.ma = mat_a; R.ms = mat_sigma; R.mm = mat_m;
    R.emit = (int*)malloc(sizeof(int) * (size_t)(S->T > 0 ? S->T : 1));
    R.cdf = (double*)malloc(sizeof(double) * (size_t)(S->T > 0 ? S->T : 1));
    R.n_emit = 0;
    R.A = 0.0;
    for (int64_t t = 0; t < S->T; ++t)
        if (is_emitter(S, (int)t)) {
            R.A += 0.5 * S->tri[t].area2;
            R.emit[R.n_emit] = (int)t;
            R.cdf[R.n_emit] = R.A;
            R.n_emit++;
        }
    R.qx = qx; R.qn = qn; R.qwo = qwo; R.qtri = qtri; R.N = N;
    R.seed = seed; R.request_id = request_id; R.point_base = point_base;
    R.spp_d = spp_d; R.spp_s = spp_s; R.K = K; R.sigma = sigma;
    R.sigma_c = sigma_c; R.max_depth = max_depth; R.mis = mis; R.eta = eta;
    R.out = out; R.per_sample = per_sample; R.amb = amb;
    R.ps_lo = (eta > 0 && per_sample) ? ps_lo : NULL;
    R.ps_hi = R.ps_lo ? ps_hi : NULL;
    R.unb = R.ps_lo ? unb : NULL;
    R.smax = spp_d > spp_s ? spp_d : spp_s;
    R.next = 0;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, refine_worker, &R);
    refine_worker(&R);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
    free(R.emit);
    free(R.cdf);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Emitter extraction (Sec. 4.4, Eq. 12)                                */
/* ------------------------------------------------------------------ */

/* n locations uniform on every triangle: the square-root map of two
 * uniforms (u1, u2) from the Philox words of counter (t, j, 0x400, rid)
 * gives barycentrics (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2).
 * x: [T * n][3], triangle-major. */
void oracle_emitter_points(const oscene* S, uint64_t seed, uint32_t rid, int n, double* x)
{
    for (int64_t t = 0; t < S->T; ++t) {
        const otri* tr = &S->tri[t];
        for (int j = 0; j < n; ++j) {
            double u[4];
            philox_words((uint32_t)t, (uint32_t)j, 0x400u, rid, seed, u);
            double r1 = sqrt(u[0]);
            double b0 = 1.0 - r1, b1 = r1 * (1.0 - u[1]), b2 = r1 * u[1];
            double* p = x + 3 * (t * n + j);
            for (int a = 0; a < 3; ++a) p[a] = b0 * tr->v0[a] + b1 * tr->v1[a] + b2 * tr->v2[a];
        }
    }
}

/* A triangle is an emitter when the mean of its n mask values is above the
 * threshold (0.01 in the paper); the sum runs in sample order in FP64. */
void oracle_emitter_classify(const float* alpha, int64_t T, int n, float thr, double* mean, uint8_t* flag)
{
    for (int64_t t = 0; t < T; ++t) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += (double)alpha[t * n + j];
        double m = s / (double)n;
        mean[t] = m;
        flag[t] = m > (double)thr;
    }
}

/* IEEE totalOrder on floats: -NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN. */
static int float_total_order(const void* pa, const void* pb)
{
    float a = *(const float*)pa, b = *(const float*)pb;
    int ca = isnan(a) ? (signbit(a) ? 0 : 2) : 1;
    int cb = isnan(b) ? (signbit(b) ? 0 : 2) : 1;
    if (ca != cb) return ca < cb ? -1 : 1;
    if (ca == 1) {
        if (a < b) return -1;
        if (a > b) return 1;
        if (signbit(a) != signbit(b)) return signbit(a) ? -1 : 1;
        return 0;
    }
    uint32_t ua, ub;
    memcpy(&ua, &a, 4);
    memcpy(&ub, &b, 4);
    if (ua == ub) return 0;
    return ((ua < ub) == (ca == 2)) ? -1 : 1;
}

/* Eq. 12 with zero reflectance at an emitter: the L1 fit of L_e to the
 * pixels whose first hit is the triangle is their per-channel median; with
 * an even count the lower of the two middle values.  Pixel p's triangle is
 * tri[p * stride] (outside [0, T): none).  Non-emitters and emitters no
 * pixel hits get 0. */
void oracle_emitter_radiance(const int32_t* tri, int64_t stride, const float* rgb, int64_t P,
                             const uint8_t* flag, int64_t T, float* Le, int32_t* count)
{
    int64_t* start = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    float* vals = (float*)malloc(sizeof(float) * (size_t)(P > 0 ? P : 1));
    int64_t* fill = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    for (int64_t t = 0; t < T; ++t) count[t] = 0;
    for (int64_t p = 0; p < P; ++p) {
        int32_t t = tri[p * stride];
        if (t >= 0 && t < T && flag[t]) count[t]++;
    }
    for (int64_t t = 0; t < T; ++t) start[t + 1] = start[t] + count[t];
    for (int c = 0; c < 3; ++c) {
        for (int64_t t = 0; t < T; ++t) fill[t] = start[t];
        for (int64_t p = 0; p < P; ++p) {
            int32_t t = tri[p * stride];
            if (t >= 0 && t < T && flag[t]) vals[fill[t]++] = rgb[3 * p + c];
        }
        for (int64_t t = 0; t < T; ++t) {
            if (count[t] == 0) { Le[3 * t + c] = 0.0f; continue; }
            qsort(vals + start[t], (size_t)count[t], sizeof(float), float_total_order);
            Le[3 * t + c] = vals[start[t] + (count[t] - 1) / 2];
        }
    }
    free(start);
    free(vals);
    free(fill);
}

/* ------------------------------------------------------------------ */
/* The BRDF of Eq. 1 as the refinement evaluates it                      */
/* ------------------------------------------------------------------ */

/* f[c] = f_r(wo, wi)[c] * (n . wi) for one material (albedo, roughness,
 * metallic), the product the refinement's path vertices use; exposed so
 * that its symmetry (f_r(wo, wi) = f_r(wi, wo)) can be checked. */
void oracle_brdf_cos(const double* n, const double* wo, const double* wi, const float* albedo,
                     float sigma, float metal, double* f)
{
    refine_job R;
    memset(&R, 0, sizeof(R));
    R.ma = albedo;
    R.ms = &sigma;
    R.mm = &metal;
    double pdf, Pd;
    int amb = 0;
    vertex_brdf_h(&R, 0, n, wo, wi, NULL, f, &pdf, &Pd, &amb);
}
