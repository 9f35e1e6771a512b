"""FP64 CPU oracle for the factorized shading-term bake (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
path never imports, links or executes anything here, and this package never
imports the CUDA path.  The two share only the seeded input generators of
``workloads/``.

Contents (each function cites the passage it restates):

* ``fipt_oracle.c`` (compiled by :func:`build`): Philox4x32-10, the bake of
  Eq. 6-7 through the one-segment cache query of Eq. 9, closest hit (brute
  force and an independent spatial-median BVH), pinhole first hits, Morton
  codes and the binary radix tree, the voxel radiance cache, and emitter
  extraction (sampling, mask classification, the median of Eq. 12).
* this module: ctypes bindings, plus the factorized render of Eq. 5 with the
  roughness lerp of Eq. 8, the tone-mapped loss of Eq. 14, its analytic
  gradient, and the per-triangle rendering error of Sec. 4.4.

Ambiguous hits.  The CUDA path intersects in float32, the oracle in float64.
Where several hits are correct for a float32 ray (the ray passes within
rounding of a triangle edge, two triangles lie at nearly the same distance,
or a hit is grazing so its facing is within rounding), the oracle reports
the whole set: with ``eta > 0`` a triangle is a candidate when the ray meets
its plane with every in-plane edge distance >= -eta*(L+t)/max(|cos|, 0.05)
and t > -eta*(L+t), and its t is not beyond the closest hit that is certain
(edge distances >= +eta*(L+t)/max(|cos|,0.05)); a miss is a candidate when no
hit is certain.  L is the scene's largest extent.  Bake bounds ``lo``/``hi``
take, per ray, the minimum / maximum incident radiance over the candidates.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, quadrature, brute force, published test vectors,
invariants), except agreement with the paper's own Mitsuba bakes, for which
no data exists (parity with the paper's images unpinned).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fipt_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

MAXC = 24  # candidate slots per ray, must match OMAXC in fipt_oracle.c


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain C11, pthreads, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                               "-ffp-contract=off", "-fno-fast-math",
                               _SRC, "-o", tmp, "-lm", "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


def _L():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_OUT)
        P, I64, I32, D, U64, U32 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32)
        L.oracle_philox4x32_10.argtypes = [P, P, I64, P]
        L.oracle_strat_uv.argtypes = [ctypes.c_int, P, P, P, I64, P, P]
        L.oracle_scene_create.argtypes = [P, I64, P, I64, P, P]
        L.oracle_scene_create.restype = P
        L.oracle_scene_destroy.argtypes = [P]
        L.oracle_scene_info.argtypes = [P, P, P, P, P]
        L.oracle_closest.argtypes = [P, P, P, I64, P, D, I32, P, P, P, P, P, P, P]
        L.oracle_closest.restype = I32
        L.oracle_bake.argtypes = [P, P, P, P, P, I64, U64, U32, U32, I32, I32, I32, P,
                                  D, I32, P, P, P, P]
        L.oracle_camera_queries.argtypes = [P, P, I32, I32, I32, P, I64, D, P, P, P, P,
                                            P, P, P]
        L.oracle_camera_queries.restype = I32
        L.oracle_refine.argtypes = [P, P, P, P, P, P, P, P, I64, U64, U32, U32, I32, I32, I32, P,
                                    D, I32, I32, D, I32, P, P, P, P, P, P]
        L.oracle_scene_set_environment.argtypes = [P, P, I32, I32]
        L.oracle_env_lookup.argtypes = [P, P, I64, P]
        L.oracle_voxel_pool.argtypes = [P, P, P, I64, I32, P]
        L.oracle_scene_set_voxel_cache.argtypes = [P, P, I32]
        L.oracle_brdf_cos.argtypes = [P, P, P, P, ctypes.c_float, ctypes.c_float, P]
        L.oracle_emitter_points.argtypes = [P, U64, U32, I32, P]
        L.oracle_emitter_classify.argtypes = [P, I64, I32, ctypes.c_float, P, P]
        L.oracle_emitter_radiance.argtypes = [P, I64, P, I64, P, I64, P, P]
        L.oracle_morton.argtypes = [P, I64, P, I64, P]
        L.oracle_radix_tree.argtypes = [P, P, I64, P, P, P, P]
        L.oracle_radix_tree.restype = I32
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- RNG
def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11).  ctr [n,4] u32, key [n,2] u32."""
    ctr = _c(ctr, np.uint32).reshape(-1, 4)
    key = _c(key, np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    _L().oracle_philox4x32_10(_p(ctr), _p(key), len(ctr), _p(out))
    return out


def strat_uv(S, s, r1, r2):
    """The jittered stratification of a (point, lobe) pair's S lobe samples:
    sample s in cell (s mod nx, s div nx) of an nx x ny grid over (u1, u2),
    placed by its uniforms (r1, r2) -> (u1, u2)."""
    s = _c(s, np.uint32).ravel()
    r1 = _c(r1, np.float64).ravel()
    r2 = _c(r2, np.float64).ravel()
    u1 = np.empty_like(r1)
    u2 = np.empty_like(r2)
    _L().oracle_strat_uv(int(S), _p(s), _p(r1), _p(r2), len(s), _p(u1), _p(u2))
    return u1, u2


def uniforms24(words):
    """u = (w >> 8) * 2^-24: the top 24 bits of a Philox word in [0, 1)."""
    return (np.asarray(words, np.uint32) >> 8).astype(np.float64) * 2.0 ** -24


# ---------------------------------------------------------------- scene
class OracleScene:
    """A triangle mesh held in FP64 with its own spatial-median BVH."""

    def __init__(self, V, F, Le=None, cache=None):
        self.V = _c(V, np.float32)
        self.F = _c(F, np.int32)
        self.T = len(self.F)
        self.Le = _c(Le if Le is not None else np.zeros((self.T, 3)), np.float32)
        self.cache = _c(cache if cache is not None else np.zeros((self.T, 3)), np.float32)
        self._h = _L().oracle_scene_create(_p(self.V), len(self.V), _p(self.F), self.T,
                                           _p(self.Le), _p(self.cache))
        lo = np.zeros(3)
        hi = np.zeros(3)
        eps = np.zeros(1)
        L = np.zeros(1)
        _L().oracle_scene_info(self._h, _p(lo), _p(hi), _p(eps), _p(L))
        self.lo, self.hi, self.eps, self.L = lo, hi, float(eps[0]), float(L[0])

    @classmethod
    def from_mesh(cls, m):
        return cls(m.V, m.F, m.Le, m.cache)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.oracle_scene_destroy(self._h)
            self._h = None

    def set_environment(self, env):
        """Equirectangular environment radiance [H, W, 3] for rays that miss
        (None clears it); see env_lookup in fipt_oracle.c for the mapping."""
        if env is None:
            _L().oracle_scene_set_environment(self._h, None, 0, 0)
            self._env = None
            return
        self._env = _c(env, np.float32)
        H, W = self._env.shape[:2]
        _L().oracle_scene_set_environment(self._h, _p(self._env), int(W), int(H))

    def env_lookup(self, dirs):
        """Environment radiance [n, 3] seen along unit directions dirs [n, 3]
        (zero without a map)."""
        d = _c(dirs, np.float64).reshape(-1, 3)
        out = np.zeros((len(d), 3))
        _L().oracle_env_lookup(self._h, _p(d), len(d), _p(out))
        return out

    def voxel_pool(self, x, L, R):
        """Sec. 4.2: average pooling of pixel radiance L [P,3] at first-hit
        points x [P,3] onto an R^3 grid over the scene box -> [R,R,R,4]
        (mean rgb, count), index [z][y][x]."""
        x = _c(x, np.float32)
        L = _c(L, np.float32)
        out = np.zeros((R, R, R, 4))
        _L().oracle_voxel_pool(self._h, _p(x), _p(L), len(x), int(R), _p(out))
        return out

    def set_voxel_cache(self, grid):
        """Use a pooled grid as the cache L' (None: per-triangle values)."""
        if grid is None:
            _L().oracle_scene_set_voxel_cache(self._h, None, 0)
            return
        g = _c(grid, np.float64)
        _L().oracle_scene_set_voxel_cache(self._h, _p(g), int(g.shape[0]))

    def emitter_points(self, n_per_tri=100, seed=0, request_id=0):
        """Sec. 4.4: n_per_tri uniform locations on every triangle (FP64,
        [T * n_per_tri, 3], triangle-major), Philox counter (t, j, 0x400, rid)."""
        out = np.zeros((self.T * int(n_per_tri), 3))
        _L().oracle_emitter_points(self._h, int(seed), int(request_id), int(n_per_tri), _p(out))
        return out

    def closest(self, orig, dirs, skip=None, eta=0.0, brute=False):
        """Closest hit of rays (o + t d, t > 0), ties by (t, id); FP64 MT."""
        o = _c(orig, np.float64).reshape(-1, 3)
        d = _c(dirs, np.float64).reshape(-1, 3)
        n = len(o)
        sk = None if skip is None else _c(skip, np.int32)
        hid = np.empty(n, np.int32)
        ht = np.empty(n, np.float64)
        hf = np.empty(n, np.int32)
        cid = np.full((n, MAXC), -1, np.int32)
        ct = np.full((n, MAXC), np.inf)
        nc = np.zeros(n, np.int32)
        mp = np.zeros(n, np.int32)
        _L().oracle_closest(self._h, _p(o), _p(d), n, _p(sk), float(eta), int(brute),
                            _p(hid), _p(ht), _p(hf), _p(cid), _p(ct), _p(nc), _p(mp))
        return {"id": hid, "t": ht, "front": hf.astype(bool), "cand_id": cid,
                "cand_t": ct, "n_cand": nc, "miss_possible": mp.astype(bool)}

    def bake(self, q, sigma, spp_d, spp_s=None, seed=0, request_id=0, point_base=0,
             eta=0.0, nthreads=None):
        """Eq. 6-7 estimated as in Sec. 6 (stage 1) with the cache query of Eq. 9.

        Returns dict with ``Ld`` [N,3], ``Ls0`` [N,K,3], ``Ls1`` [N,K,3] (the
        nominal estimate) and, when eta > 0, ``lo``/``hi`` versions and the
        per-point count of ambiguous rays ``n_amb``.
        """
        spp_s = spp_d if spp_s is None else spp_s
        sig = _c(sigma, np.float64)
        K = len(sig)
        x, nn, wo, tri = (_c(q["x"], np.float32), _c(q["n"], np.float32),
                          _c(q["wo"], np.float32), _c(q["tri"], np.int32))
        N = len(x)
        W = 3 + 6 * K
        nom = np.zeros((N, W))
        lo = np.zeros((N, W)) if eta > 0 else None
        hi = np.zeros((N, W)) if eta > 0 else None
        namb = np.zeros(N, np.int64)
        _L().oracle_bake(self._h, _p(x), _p(nn), _p(wo), _p(tri), N, int(seed) & (2**64 - 1),
                         int(request_id), int(point_base), int(spp_d), int(spp_s), K, _p(sig),
                         float(eta), int(nthreads or default_threads()), _p(nom), _p(lo),
                         _p(hi), _p(namb))

        def split(a):
            return {"Ld": a[:, :3], "Ls0": a[:, 3:3 + 3 * K].reshape(N, K, 3),
                    "Ls1": a[:, 3 + 3 * K:].reshape(N, K, 3)}
        out = split(nom)
        out["flat"] = nom
        if eta > 0:
            out["lo"] = lo
            out["hi"] = hi
            out["n_amb"] = namb
        return out

    def refine(self, q, sigma, spp_d, spp_s, albedo, rough, metal, sigma_c=0.6, max_depth=8,
               mis=True, seed=0, request_id=0, point_base=0, eta=0.0, per_sample=False,
               bounds=False, nthreads=None):
        """Stage-3 path-traced shadings (Sec. 4.3, Eq. 10; MIS per Sec. 6) with
        per-triangle materials albedo [T,3], rough [T], metal [T].  Returns the
        bake layout; with per_sample also every sample's 6 values
        ([N, 1+K, Smax, 6]) and its ambiguity flag ([N, 1+K, Smax]).  With
        bounds (needs per_sample and eta > 0) also ``lo`` / ``hi``, each
        sample's range over every decision a float32 path may take the other
        way, and ``unbounded`` ([N, 1+K, Smax] bool) where that range is
        [0, inf].  The roughness threshold is rounded to float32 first:
        materials are float32, so "rougher than sigma_c" is decided on
        float32 values."""
        sig = _c(sigma, np.float64)
        K = len(sig)
        x, nn, wo, tri = (_c(q["x"], np.float32), _c(q["n"], np.float32),
                          _c(q["wo"], np.float32), _c(q["tri"], np.int32))
        a, r, m = _c(albedo, np.float32), _c(rough, np.float32), _c(metal, np.float32)
        N = len(x)
        W = 3 + 6 * K
        out = np.zeros((N, W))
        smax = max(spp_d, spp_s)
        ps = np.zeros((N, K + 1, smax, 6)) if per_sample else None
        amb = np.zeros((N, K + 1, smax), np.uint8) if per_sample else None
        bounds = bool(bounds and per_sample and eta > 0)
        lo = np.zeros((N, K + 1, smax, 6)) if bounds else None
        hi = np.zeros((N, K + 1, smax, 6)) if bounds else None
        unb = np.zeros((N, K + 1, smax), np.uint8) if bounds else None
        _L().oracle_refine(self._h, _p(a), _p(r), _p(m), _p(x), _p(nn), _p(wo), _p(tri), N,
                           int(seed) & (2**64 - 1), int(request_id), int(point_base), int(spp_d),
                           int(spp_s), K, _p(sig), float(np.float32(sigma_c)), int(max_depth),
                           int(bool(mis)),
                           float(eta), int(nthreads or default_threads()), _p(out), _p(ps), _p(amb),
                           _p(lo), _p(hi), _p(unb))
        res = {"Ld": out[:, :3], "Ls0": out[:, 3:3 + 3 * K].reshape(N, K, 3),
               "Ls1": out[:, 3 + 3 * K:].reshape(N, K, 3), "flat": out}
        if per_sample:
            res["per_sample"] = ps
            res["amb"] = amb.astype(bool)
        if bounds:
            res["lo"], res["hi"], res["unbounded"] = lo, hi, unb.astype(bool)
        return res

    def camera_queries(self, cams, W, H, pixels, eta=0.0):
        """First hits of pinhole pixels (row layout as oracle_camera_queries)."""
        cams = _c(cams, np.float32).reshape(-1, 10)
        pix = _c(pixels, np.int64)
        n = len(pix)
        qx = np.zeros((n, 3))
        qn = np.zeros((n, 3))
        qwo = np.zeros((n, 3))
        tri = np.zeros(n, np.int32)
        nc = np.zeros(n, np.int32)
        cid = np.full((n, MAXC), -1, np.int32)
        mp = np.zeros(n, np.int32)
        rc = _L().oracle_camera_queries(self._h, _p(cams), len(cams), int(W), int(H), _p(pix),
                                        n, float(eta), _p(qx), _p(qn), _p(qwo), _p(tri),
                                        _p(nc), _p(cid), _p(mp))
        if rc != 0:
            raise ValueError("pixel index out of range")
        return {"x": qx, "n": qn, "wo": qwo, "tri": tri, "n_cand": nc, "cand_id": cid,
                "miss_possible": mp.astype(bool)}


# ---------------------------------------------------------------- LBVH targets
def morton_codes(V, F):
    """63-bit Morton codes of triangle box centres (FP64 quantisation)."""
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    codes = np.zeros(len(F), np.uint64)
    _L().oracle_morton(_p(V), len(V), _p(F), len(F), _p(codes))
    return codes


def lbvh_reference(V, F):
    """Bit-exact LBVH targets: codes, stable order, radix-tree nodes, boxes.

    The order is the stable sort of (code, triangle index).  Internal nodes
    are listed as (first, last, split) over positions in that order; a node
    box is the float min/max over the boxes of its triangles.
    """
    V = _c(V, np.float32)
    F = _c(F, np.int32)
    codes = morton_codes(V, F)
    order = np.lexsort((np.arange(len(F)), codes)).astype(np.int32)
    sc = np.ascontiguousarray(codes[order])
    tv = V[F[order]]                                   # [T,3 verts,3]
    tbox = np.ascontiguousarray(np.concatenate([tv.min(1), tv.max(1)], 1), np.float32)
    T = len(F)
    n = max(T - 1, 0)
    first = np.zeros(n, np.int32)
    last = np.zeros(n, np.int32)
    split = np.zeros(n, np.int32)
    nbox = np.zeros((n, 6), np.float32)
    if T >= 2:
        got = _L().oracle_radix_tree(_p(sc), _p(tbox), T, _p(first), _p(last), _p(split),
                                     _p(nbox))
        assert got == T - 1
    return {"codes": codes, "order": order, "sorted_codes": sc, "first": first,
            "last": last, "split": split, "node_box": nbox, "tri_box": tbox}


# ---------------------------------------------------------------- render (Eq. 5, 8, 14)
def tonemap(x):
    """Gamma of Eq. 14 (Munkberg et al. 2022): sRGB transfer curve applied
    to log(1 + max(x, 0))."""
    y = np.log1p(np.maximum(np.asarray(x, np.float64), 0.0))
    return np.where(y <= 0.0031308, 12.92 * y,
                    1.055 * np.power(np.maximum(y, 0.0031308), 1.0 / 2.4) - 0.055)


def tonemap_grad(x):
    """d Gamma / dx (right derivative at the kinks; 0 for x < 0)."""
    x = np.asarray(x, np.float64)
    y = np.log1p(np.maximum(x, 0.0))
    ds = np.where(y <= 0.0031308, 12.92,
                  (1.055 / 2.4) * np.power(np.maximum(y, 0.0031308), 1.0 / 2.4 - 1.0))
    return np.where(x < 0.0, 0.0, ds / (1.0 + np.maximum(x, 0.0)))


def lerp_segment(rough, grid):
    """Eq. 8: segment i (largest i <= K-2 with grid[i] <= sigma after
    clamping sigma to the grid), weight t, and whether sigma was clamped."""
    grid = np.asarray(grid, np.float64)
    if len(grid) < 2:
        raise ValueError("the lerp of Eq. 8 needs at least two roughness nodes")
    r = np.asarray(rough, np.float64)
    s = np.clip(r, grid[0], grid[-1])
    i = np.clip(np.searchsorted(grid, s, side="right") - 1, 0, len(grid) - 2)
    t = (s - grid[i]) / (grid[i + 1] - grid[i])
    clamped = (r < grid[0]) | (r > grid[-1])
    return i, t, clamped


def render_forward(Ld, Ls0, Ls1, grid, albedo, rough, metal, Lgt=None, mask=None):
    """Eq. 5: L_r = k_d L_d + k_s L_s0(sigma) + L_s1(sigma), k_d = a(1-m),
    k_s = 0.04(1-m) + a m (Eq. 1), L_s* lerped over the grid (Eq. 8).
    Loss of Eq. 14 with alpha = 0: sum over valid points and channels of
    (Gamma(L_r) - Gamma(L_gt))^2."""
    Ld, Ls0, Ls1 = (np.asarray(a, np.float64) for a in (Ld, Ls0, Ls1))
    a = np.asarray(albedo, np.float64)
    m = np.asarray(metal, np.float64)[:, None]
    i, t, _ = lerp_segment(rough, grid)
    n = np.arange(len(Ld))
    S0 = (1 - t)[:, None] * Ls0[n, i] + t[:, None] * Ls0[n, i + 1]
    S1 = (1 - t)[:, None] * Ls1[n, i] + t[:, None] * Ls1[n, i + 1]
    kd = a * (1 - m)
    ks = 0.04 * (1 - m) + a * m
    Lr = kd * Ld + ks * S0 + S1
    loss = None
    if Lgt is not None:
        diff = tonemap(Lr) - tonemap(np.asarray(Lgt, np.float64))
        valid = np.ones(len(Lr), bool) if mask is None else np.asarray(mask).astype(bool)
        loss = float(np.sum(diff[valid] ** 2))
    return Lr, loss


def render_grad(Ld, Ls0, Ls1, grid, albedo, rough, metal, Lgt, mask=None, grad_scale=1.0):
    """Analytic gradient of the Eq. 14 loss through Eq. 5 and Eq. 8 with
    respect to per-point albedo (3), roughness and metallic."""
    Ld, Ls0, Ls1 = (np.asarray(a, np.float64) for a in (Ld, Ls0, Ls1))
    grid = np.asarray(grid, np.float64)
    a = np.asarray(albedo, np.float64)
    m = np.asarray(metal, np.float64)[:, None]
    i, t, clamped = lerp_segment(rough, grid)
    n = np.arange(len(Ld))
    S0 = (1 - t)[:, None] * Ls0[n, i] + t[:, None] * Ls0[n, i + 1]
    S1 = (1 - t)[:, None] * Ls1[n, i] + t[:, None] * Ls1[n, i + 1]
    kd = a * (1 - m)
    ks = 0.04 * (1 - m) + a * m
    Lr = kd * Ld + ks * S0 + S1
    g = 2.0 * (tonemap(Lr) - tonemap(np.asarray(Lgt, np.float64))) * tonemap_grad(Lr)
    if mask is not None:
        g = g * np.asarray(mask).astype(bool)[:, None]
    g = g * grad_scale
    g_a = g * ((1 - m) * Ld + m * S0)
    g_m = np.sum(g * (-a * Ld + (a - 0.04) * S0), axis=1)
    w = (grid[i + 1] - grid[i])[:, None]
    dS0 = (Ls0[n, i + 1] - Ls0[n, i]) / w
    dS1 = (Ls1[n, i + 1] - Ls1[n, i]) / w
    g_s = np.sum(g * (ks * dS0 + dS1), axis=1)
    g_s = np.where(clamped, 0.0, g_s)
    return g_a, g_s, g_m


# ---------------------------------------------------------------- emitter detection
def tri_error(tri, Lr, Lgt, T):
    """Sec. 4.4: per-triangle rendering error.  err[t] = sum over pixels whose
    first hit is t of ||L_r - L_gt||^2 (linear radiance), count[t] = #pixels;
    pixels with tri < 0 (no hit) are ignored."""
    tri = np.asarray(tri)
    e = np.sum((np.asarray(Lr, np.float64) - np.asarray(Lgt, np.float64)) ** 2, axis=1)
    v = tri >= 0
    err = np.bincount(tri[v], weights=e[v], minlength=T)[:T]
    cnt = np.bincount(tri[v], minlength=T)[:T].astype(np.int32)
    return err, cnt


def emitter_classify(alpha, n_per_tri=100, threshold=0.01):
    """Sec. 4.4: emitter when the mean of a triangle's n_per_tri mask values
    exceeds the threshold.  Returns (flag u8 [T], mean f64 [T])."""
    a = _c(alpha, np.float32).reshape(-1)
    T = a.size // int(n_per_tri)
    mean = np.zeros(T)
    flag = np.zeros(T, np.uint8)
    _L().oracle_emitter_classify(_p(a), T, int(n_per_tri), float(threshold), _p(mean), _p(flag))
    return flag, mean


def emitter_radiance(tri, rgb, flag, tri_stride=1):
    """Eq. 12 with zero reflectance at emitters: per-channel lower median of
    the pixels hitting each emitter triangle.  Returns (Le f32 [T,3], count)."""
    tri = _c(tri, np.int32).reshape(-1)
    rgb = _c(rgb, np.float32).reshape(-1, 3)
    flag = _c(flag, np.uint8)
    T = len(flag)
    P = len(rgb)
    assert tri.size >= (P - 1) * tri_stride + 1 if P else True
    Le = np.zeros((T, 3), np.float32)
    cnt = np.zeros(T, np.int32)
    _L().oracle_emitter_radiance(_p(tri), int(tri_stride), _p(rgb), P, _p(flag), T, _p(Le), _p(cnt))
    return Le, cnt


def brdf_cos(n, wo, wi, albedo, sigma, metal):
    """Eq. 1's BRDF times (n . wi), as the refinement evaluates it at a path
    vertex: diffuse k_d / pi plus GGX with the Fresnel split of Eq. 7
    (k_s F0 + F1), k_d = a (1 - m), k_s = 0.04 (1 - m) + a m.  -> [3]."""
    f = np.zeros(3)
    _L().oracle_brdf_cos(_p(_c(n, np.float64)), _p(_c(wo, np.float64)), _p(_c(wi, np.float64)),
                         _p(_c(albedo, np.float32)), float(sigma), float(metal), _p(f))
    return f
