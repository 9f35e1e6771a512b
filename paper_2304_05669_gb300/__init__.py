"""GB300 bake of the factorized shading terms of Factorized Inverse Path
Tracing (Wu et al., ICCV 2023) -- Python binding of libfipt.so.

Everything here marshals torch CUDA tensors into the C ABI of
``include/fipt.h``; every step of the computation runs in the library's
sm_103a kernels.  PyTorch supplies device memory and streams only.

Queries are float32 tensors [N, 10]: x (3), n (3), wo (3) and the triangle
index stored as int32 bits in column 9 -- the 40-byte ``fipt_query``.
"""
from __future__ import annotations

import ctypes

import torch

from ._native import (BakeParams, FiptError, FIPT_MAX_K, Request, ServerStats, check, lib,
                      library_path)

__all__ = ["Context", "Scene", "bake", "bake_refine", "render_fwd", "render_bwd", "render_fwd_grad",
           "render_grad_scale", "FactorizedRender",
           "factorized_render_loss", "tri_error", "compact_queries", "pack_queries",
           "unpack_queries", "philox", "emitter_classify", "emitter_radiance", "extract_emitters",
           "FiptError", "library_path", "context", "Server"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    return t.contiguous()


def _need(t, dtype, name, shape):
    """A CUDA tensor of this dtype and exact shape (contiguous; copied if not)."""
    t = _dev(t, dtype, name)
    if tuple(t.shape) != tuple(int(d) for d in shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t


def _host(t, dtype, name, shape):
    """A CPU tensor of this dtype and exact shape (contiguous; copied if not)."""
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a CPU tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(int(d) for d in shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.contiguous()


def _queries(q, name="q"):
    q = _dev(q, torch.float32, name)
    if q.dim() != 2 or q.shape[1] != 10:
        raise ValueError("%s must be [N, 10] query records, got %s" % (name, tuple(q.shape)))
    return q


def _workspace(nbytes, device):
    """A byte tensor whose data pointer is 256-byte aligned."""
    buf = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf, buf[off:off + int(nbytes)]


class Context:
    """A library context on one CUDA device (holds the device status word)."""

    def __init__(self, device: int = 0):
        lib()
        h = ctypes.c_void_p()
        check(lib().fipt_ctx_create(int(device), ctypes.byref(h)))
        self.handle = h
        self.device = int(device)

    def sync_status(self, stream=None) -> int:
        """Waits for the stream; returns the kernels' status bits (raises if set)."""
        code = ctypes.c_int32(0)
        st = lib().fipt_sync_status(self.handle, _stream(stream), ctypes.byref(code))
        if st != 0:
            raise FiptError(st, lib().fipt_last_error().decode())
        return code.value

    def close(self):
        if getattr(self, "handle", None):
            lib().fipt_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts: dict = {}


def context(device: int | None = None) -> Context:
    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _contexts:
        _contexts[d] = Context(d)
    return _contexts[d]


def pack_queries(x, n, wo, tri):
    """[N,3] x, n, wo (float32) and [N] tri (int32) -> [N,10] query tensor."""
    N = x.shape[0]
    q = torch.empty((N, 10), dtype=torch.float32, device=x.device)
    q[:, 0:3] = x
    q[:, 3:6] = n
    q[:, 6:9] = wo
    q[:, 9:10].view(torch.int32)[:, 0] = tri.to(torch.int32)
    return q


def unpack_queries(q):
    return {"x": q[:, 0:3], "n": q[:, 3:6], "wo": q[:, 6:9],
            "tri": q[:, 9:10].contiguous().view(torch.int32)[:, 0]}


OPTIMIZE_PASSES = 2      # treelet-restructuring passes a Scene gets by default ...
OPTIMIZE_MIN_TRIS = 4096  # ... from this many triangles (smaller trees stay cache-resident)
OPTIMIZE_PASSES_LARGE = 3  # ... and from OPTIMIZE_LARGE_TRIS on: on a 2M-triangle floor
OPTIMIZE_LARGE_TRIS = 1 << 20  # a third pass (7 ms) saves 1.5 % of the node visits per ray
RELAYOUT = True           # depth-first node renumbering after the passes


class Scene:
    """A triangle mesh with its device-built LBVH (``fipt_scene_create``),
    then ``optimize`` treelet-restructuring passes (``fipt_scene_optimize``;
    0 keeps the radix tree as built; by default OPTIMIZE_PASSES for scenes
    of at least OPTIMIZE_MIN_TRIS triangles, OPTIMIZE_PASSES_LARGE from
    OPTIMIZE_LARGE_TRIS) and, after them, a depth-first
    renumbering of the nodes (``fipt_scene_relayout``; ``relayout=False``
    skips it)."""

    def __init__(self, V, F, Le, cache, ctx: Context | None = None, stream=None, optimize=None,
                 relayout=None):
        V = _dev(V, torch.float32, "V")
        F = _dev(F, torch.int32, "F")
        Le = _dev(Le, torch.float32, "Le")
        cache = _dev(cache, torch.float32, "cache")
        self.ctx = ctx or context(V.device.index)
        self.device = V.device
        self.T = int(F.shape[0])
        self.nV = int(V.shape[0])
        nbytes = ctypes.c_size_t()
        check(lib().fipt_scene_workspace_size(self.nV, self.T, ctypes.byref(nbytes)))
        self._buf, self.workspace = _workspace(nbytes.value, V.device)
        h = ctypes.c_void_p()
        check(lib().fipt_scene_create(self.ctx.handle, _ptr(V), self.nV, _ptr(F), self.T, _ptr(Le),
                                      _ptr(cache), _ptr(self.workspace), nbytes.value,
                                      _stream(stream), ctypes.byref(h)))
        self.handle = h
        self._keep = (V, F, Le, cache)    # alive until the stream has consumed them
        if optimize is None:
            optimize = (OPTIMIZE_PASSES_LARGE if self.T >= OPTIMIZE_LARGE_TRIS else
                        OPTIMIZE_PASSES if self.T >= OPTIMIZE_MIN_TRIS else 0)
        optimize = int(optimize)
        self.optimized = optimize
        if optimize:
            check(lib().fipt_scene_optimize(h, int(optimize), _stream(stream)))
            if RELAYOUT if relayout is None else relayout:
                check(lib().fipt_scene_relayout(h, _stream(stream)))

    @classmethod
    def from_mesh(cls, mesh, device="cuda", **kw):
        t = lambda a: torch.from_numpy(a).to(device)
        return cls(t(mesh.V), t(mesh.F), t(mesh.Le), t(mesh.cache), **kw)

    def info(self, stream=None):
        T = ctypes.c_int64()
        eps = ctypes.c_float()
        lo = (ctypes.c_float * 3)()
        hi = (ctypes.c_float * 3)()
        check(lib().fipt_scene_info(self.handle, _stream(stream), ctypes.byref(T), ctypes.byref(eps),
                                    lo, hi))
        return {"T": T.value, "eps": eps.value, "lo": list(lo), "hi": list(hi)}

    def set_cache(self, cache, stream=None):
        cache = _dev(cache, torch.float32, "cache")
        check(lib().fipt_scene_set_cache(self.handle, _ptr(cache), _stream(stream)))
        self._keep = self._keep + (cache,)

    def set_environment(self, env):
        """Environment radiance [H, W, 3] (CUDA float32) seen by rays that miss;
        None clears it."""
        if env is None:
            check(lib().fipt_scene_set_environment(self.handle, None, 0, 0))
            self._env = None
            return
        env = _dev(env, torch.float32, "env")
        check(lib().fipt_scene_set_environment(self.handle, _ptr(env), env.shape[1], env.shape[0]))
        self._env = env

    def voxel_cache(self, x, L, R=256, stream=None):
        """Sec. 4.2: pools pixel radiance L [P,3] at first-hit points x ([P,3],
        or [P,10] query records) onto an R^3 grid -> [R,R,R,4] (mean rgb, count)."""
        x = _dev(x, torch.float32, "x")
        L = _dev(L, torch.float32, "L")
        stride = 10 if (x.dim() == 2 and x.shape[1] == 10) else 3
        P = x.shape[0]
        nbytes = ctypes.c_size_t()
        check(lib().fipt_voxel_cache_workspace_size(P, ctypes.byref(nbytes)))
        _b, ws = _workspace(nbytes.value, x.device)
        grid = torch.empty((R, R, R, 4), dtype=torch.float32, device=x.device)
        check(lib().fipt_voxel_cache_build(self.handle, _ptr(x), stride, _ptr(L), P, int(R), _ptr(grid),
                                           _ptr(ws), nbytes.value, _stream(stream)))
        return grid

    def set_voxel_cache(self, grid):
        """Use a pooled grid as the cache L' (None: per-triangle values)."""
        if grid is None:
            check(lib().fipt_scene_set_voxel_cache(self.handle, None, 0))
            self._vox = None
            return
        grid = _dev(grid, torch.float32, "grid")
        check(lib().fipt_scene_set_voxel_cache(self.handle, _ptr(grid), grid.shape[0]))
        self._vox = grid

    def set_emission(self, Le, stream=None):
        """Replaces L_e [T,3] (rebuilds the emitter table, keeps the BVH)."""
        Le = _dev(Le, torch.float32, "Le")
        check(lib().fipt_scene_set_emission(self.handle, _ptr(Le), _stream(stream)))
        self._keep = self._keep + (Le,)

    def emitter_points(self, n_per_tri=100, seed=0, request_id=0, stream=None):
        """Sec. 4.4: n_per_tri uniform locations on every triangle -> f32
        [T * n_per_tri, 3] (triangle-major), where the emission mask is read."""
        x = torch.empty((self.T * int(n_per_tri), 3), dtype=torch.float32, device=self.device)
        check(lib().fipt_emitter_sample_points(self.handle, int(seed), int(request_id), int(n_per_tri),
                                               _ptr(x), _stream(stream)))
        return x

    def set_materials(self, albedo, rough, metal, stream=None):
        """Per-triangle albedo [T,3], roughness [T], metallic [T] (refinement)."""
        albedo = _dev(albedo, torch.float32, "albedo")
        rough = _dev(rough, torch.float32, "rough")
        metal = _dev(metal, torch.float32, "metal")
        check(lib().fipt_scene_set_materials(self.handle, _ptr(albedo), _ptr(rough), _ptr(metal),
                                             _stream(stream)))
        self._keep = self._keep + (albedo, rough, metal)

    def export(self, stream=None):
        T = self.T
        ni = max(T - 1, 1 if T == 1 else 0)
        d = self.device
        out = {"morton": torch.empty(T, dtype=torch.int64, device=d),
               "order": torch.empty(T, dtype=torch.int32, device=d),
               "box": torch.empty((ni, 6), dtype=torch.float32, device=d),
               "child": torch.empty((ni, 2), dtype=torch.int32, device=d)}
        if not self.optimized:
            out["range"] = torch.empty((ni, 3), dtype=torch.int32, device=d)
        check(lib().fipt_scene_debug_export(self.handle, _ptr(out["morton"]), _ptr(out["order"]),
                                            _ptr(out.get("range")), _ptr(out["box"]), _ptr(out["child"]),
                                            _stream(stream)))
        return out

    def trace(self, orig, dirs, skip=None, stream=None):
        """Closest hits: (tri int32, t float32, front int32) per ray."""
        orig = _dev(orig, torch.float32, "orig")
        dirs = _dev(dirs, torch.float32, "dirs")
        n = orig.shape[0]
        skip = None if skip is None else _dev(skip, torch.int32, "skip")
        tri = torch.empty(n, dtype=torch.int32, device=orig.device)
        t = torch.empty(n, dtype=torch.float32, device=orig.device)
        fr = torch.empty(n, dtype=torch.int32, device=orig.device)
        check(lib().fipt_trace_closest(self.handle, _ptr(orig), _ptr(dirs), n, _ptr(skip), _ptr(tri),
                                       _ptr(t), _ptr(fr), _stream(stream)))
        return tri, t, fr

    def camera_queries(self, cams, W, H, stream=None, out=None, valid=None):
        cams = _dev(cams, torch.float32, "cams")
        P = cams.shape[0] * W * H
        if out is None:
            out = torch.empty((P, 10), dtype=torch.float32, device=cams.device)
        if valid is None:
            valid = torch.empty(P, dtype=torch.int32, device=cams.device)
        check(lib().fipt_camera_queries(self.handle, _ptr(cams), cams.shape[0], int(W), int(H),
                                        _ptr(out), _ptr(valid), _stream(stream)))
        return out, valid

    def close(self):
        if getattr(self, "handle", None):
            lib().fipt_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compact_queries(q, valid, max_out, stream=None):
    """First ``max_out`` valid records in order -> (out, pixel_of, n_out[1] int64)."""
    q = _queries(q)
    P = q.shape[0]
    valid = _need(valid, torch.int32, "valid", (P,))
    nbytes = ctypes.c_size_t()
    check(lib().fipt_compact_workspace_size(P, ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, q.device)
    out = torch.empty((int(max_out), 10), dtype=torch.float32, device=q.device)
    pix = torch.empty(int(max_out), dtype=torch.int32, device=q.device)
    n_out = torch.empty(1, dtype=torch.int64, device=q.device)
    check(lib().fipt_compact_queries(_ptr(q), _ptr(valid), P, int(max_out), _ptr(out), _ptr(pix),
                                     _ptr(n_out), _ptr(ws), nbytes.value, _stream(stream)))
    return out, pix, n_out


def bake_params(sigma, spp_diffuse, spp_specular=None, seed=0, request_id=0, point_base=0,
                stats=None):
    p = BakeParams()
    p.seed = int(seed) & (2 ** 64 - 1)
    p.request_id = int(request_id)
    p.point_base = int(point_base)
    p.spp_diffuse = int(spp_diffuse)
    p.spp_specular = int(spp_diffuse if spp_specular is None else spp_specular)
    sig = [float(s) for s in sigma]
    if not 1 <= len(sig) <= FIPT_MAX_K:
        raise ValueError("need 1..%d roughness levels" % FIPT_MAX_K)
    p.K = len(sig)
    for k, s in enumerate(sig):
        p.sigma[k] = s
    p.stats = stats.data_ptr() if stats is not None else None
    return p


def query_order(scene: Scene, q, stream=None):
    """Indices of the query points sorted by the Morton code of their
    positions (``fipt_query_order``) -> int32 [N] on the queries' device."""
    q = _queries(q)
    N = q.shape[0]
    order = torch.empty(N, dtype=torch.int32, device=q.device)
    if N == 0:
        return order
    nbytes = ctypes.c_size_t()
    check(lib().fipt_query_order_workspace_size(N, ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, q.device)
    check(lib().fipt_query_order(scene.handle, _ptr(q), N, _ptr(order), _ptr(ws), nbytes.value, _stream(stream)))
    if stream is not None:             # the buffers outlive this call on that stream's work
        _b.record_stream(stream)
        order.record_stream(stream)
    return order


def bake(scene: Scene, q, sigma, spp_diffuse, spp_specular=None, seed=0, request_id=0,
         point_base=0, stats=None, out=None, stream=None, order=True):
    """Shading terms (Eq. 6-7) at the query points -> (Ld [N,3], Ls0 [N,K,3], Ls1 [N,K,3]).
    ``order``: True bakes the points in Morton order of their positions
    (``query_order``; faster, the same results up to the float32 caveat of
    ``fipt_bake_params.order``), False in the given order, or
    an int32 [N] CUDA permutation to use."""
    q = _queries(q)
    N = q.shape[0]
    K = len(sigma)
    if out is None:
        out = (torch.empty((N, 3), dtype=torch.float32, device=q.device),
               torch.empty((N, K, 3), dtype=torch.float32, device=q.device),
               torch.empty((N, K, 3), dtype=torch.float32, device=q.device))
    p = bake_params(sigma, spp_diffuse, spp_specular, seed, request_id, point_base, stats)
    perm = None
    if order is True:
        perm = query_order(scene, q, stream) if N > 0 else None
    elif order is not None and order is not False:
        perm = _need(order, torch.int32, "order", (N,))
    p.order = perm.data_ptr() if perm is not None else None
    if perm is not None and stream is not None:
        perm.record_stream(stream)
    check(lib().fipt_bake(scene.handle, _ptr(q), N, ctypes.byref(p), _ptr(out[0]), _ptr(out[1]),
                          _ptr(out[2]), _stream(stream)))
    return out


def bake_refine(scene: Scene, q, sigma, spp_diffuse, spp_specular=None, sigma_c=0.6, max_depth=8,
                mis=True, seed=0, request_id=0, point_base=0, per_sample=False, stats=None, stream=None):
    """Stage-3 path-traced shadings (Sec. 4.3, Eq. 10, MIS) -> (Ld, Ls0, Ls1[, per_sample]).
    ``stats``: an int64 [4] CUDA tensor that receives (added) rays, node
    visits, triangle tests and (max) the deepest stack."""
    q = _queries(q)
    N = q.shape[0]
    K = len(sigma)
    spp_s = spp_diffuse if spp_specular is None else spp_specular
    out = (torch.empty((N, 3), dtype=torch.float32, device=q.device),
           torch.empty((N, K, 3), dtype=torch.float32, device=q.device),
           torch.empty((N, K, 3), dtype=torch.float32, device=q.device))
    ps = (torch.empty((N, K + 1, max(spp_diffuse, spp_s), 6), dtype=torch.float32, device=q.device)
          if per_sample else None)
    p = bake_params(sigma, spp_diffuse, spp_s, seed, request_id, point_base, stats)
    nbytes = ctypes.c_size_t()
    check(lib().fipt_bake_refine_workspace_size(N, ctypes.byref(p), int(max_depth), ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, q.device)
    check(lib().fipt_bake_refine(scene.handle, _ptr(q), N, ctypes.byref(p), float(sigma_c),
                                 int(max_depth), int(bool(mis)), _ptr(out[0]), _ptr(out[1]),
                                 _ptr(out[2]), _ptr(ps), _ptr(ws), nbytes.value, _stream(stream)))
    return out + ((ps,) if per_sample else ())


def _grid(sigma_grid):
    g = (ctypes.c_float * len(sigma_grid))(*[float(s) for s in sigma_grid])
    return g, len(sigma_grid)


def _render_inputs(N, K, Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask):
    Ld = _need(Ld, torch.float32, "Ld", (N, 3))
    Ls0 = _need(Ls0, torch.float32, "Ls0", (N, K, 3))
    Ls1 = _need(Ls1, torch.float32, "Ls1", (N, K, 3))
    albedo = _need(albedo, torch.float32, "albedo", (N, 3))
    rough = _need(rough, torch.float32, "rough", (N,))
    metal = _need(metal, torch.float32, "metal", (N,))
    if Lgt is not None:
        Lgt = _need(Lgt, torch.float32, "Lgt", (N, 3))
    if mask is not None:
        mask = _need(mask, torch.uint8, "mask", (N,))
    return Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask


def render_fwd(Ld, Ls0, Ls1, sigma_grid, albedo, rough, metal, Lgt=None, mask=None, stream=None,
               Lr=None):
    """Eq. 5 + Eq. 8 -> Lr [N,3]; with Lgt also the Eq. 14 loss (float64 [1])."""
    N = Ld.shape[0]
    g, K = _grid(sigma_grid)
    Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask = _render_inputs(N, K, Ld, Ls0, Ls1, albedo, rough,
                                                                   metal, Lgt, mask)
    if Lr is None:
        Lr = torch.empty((N, 3), dtype=torch.float32, device=Ld.device)
    elif not (Lr.is_cuda and Lr.dtype == torch.float32 and tuple(Lr.shape) == (N, 3) and Lr.is_contiguous()):
        raise ValueError("Lr must be a contiguous CUDA float32 [N, 3] tensor")
    loss = torch.zeros(1, dtype=torch.float64, device=Ld.device) if Lgt is not None else None
    nbytes = ctypes.c_size_t()
    check(lib().fipt_render_workspace_size(N, ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, Ld.device)
    check(lib().fipt_render_fwd(_ptr(Ld), _ptr(Ls0), _ptr(Ls1), N, K, g, _ptr(albedo), _ptr(rough),
                                _ptr(metal), _ptr(Lgt), _ptr(mask), _ptr(Lr), _ptr(loss), _ptr(ws),
                                nbytes.value, _stream(stream)))
    return Lr, loss


def render_bwd(Ld, Ls0, Ls1, sigma_grid, albedo, rough, metal, Lgt, mask=None, grad_loss=None,
               stream=None):
    """d loss / d (albedo, rough, metal), scaled by grad_loss (float64 device scalar)."""
    N = Ld.shape[0]
    g, K = _grid(sigma_grid)
    if Lgt is None:
        raise ValueError("render_bwd needs Lgt")
    Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask = _render_inputs(N, K, Ld, Ls0, Ls1, albedo, rough,
                                                                   metal, Lgt, mask)
    if grad_loss is not None:
        grad_loss = _need(grad_loss, torch.float64, "grad_loss", (1,))
    ga = torch.empty((N, 3), dtype=torch.float32, device=Ld.device)
    gr = torch.empty(N, dtype=torch.float32, device=Ld.device)
    gm = torch.empty(N, dtype=torch.float32, device=Ld.device)
    check(lib().fipt_render_bwd(_ptr(Ld), _ptr(Ls0), _ptr(Ls1), N, K, g, _ptr(albedo), _ptr(rough),
                                _ptr(metal), _ptr(Lgt), _ptr(mask), _ptr(grad_loss), _ptr(ga),
                                _ptr(gr), _ptr(gm), _stream(stream)))
    return ga, gr, gm


def render_fwd_grad(Ld, Ls0, Ls1, sigma_grid, albedo, rough, metal, Lgt, mask=None, stream=None):
    """Forward, loss and gradient in one pass -> (Lr, loss, (g_albedo, g_rough, g_metal)):
    render_fwd's results and render_bwd's for grad_loss = 1, each input read once."""
    N = Ld.shape[0]
    g, K = _grid(sigma_grid)
    if Lgt is None:
        raise ValueError("render_fwd_grad needs Lgt")
    Ld, Ls0, Ls1, albedo, rough, metal, Lgt, mask = _render_inputs(N, K, Ld, Ls0, Ls1, albedo, rough,
                                                                   metal, Lgt, mask)
    Lr = torch.empty((N, 3), dtype=torch.float32, device=Ld.device)
    loss = torch.zeros(1, dtype=torch.float64, device=Ld.device)
    ga = torch.empty((N, 3), dtype=torch.float32, device=Ld.device)
    gr = torch.empty(N, dtype=torch.float32, device=Ld.device)
    gm = torch.empty(N, dtype=torch.float32, device=Ld.device)
    nbytes = ctypes.c_size_t()
    check(lib().fipt_render_workspace_size(N, ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, Ld.device)
    check(lib().fipt_render_fwd_grad(_ptr(Ld), _ptr(Ls0), _ptr(Ls1), N, K, g, _ptr(albedo), _ptr(rough),
                                     _ptr(metal), _ptr(Lgt), _ptr(mask), _ptr(Lr), _ptr(loss), _ptr(ga),
                                     _ptr(gr), _ptr(gm), _ptr(ws), nbytes.value, _stream(stream)))
    return Lr, loss, (ga, gr, gm)


def render_grad_scale(grads, grad_loss, stream=None):
    """Multiplies render_fwd_grad's gradients in place by grad_loss (float64 CUDA [1])."""
    ga, gr, gm = grads
    N = gr.shape[0]
    ga = _need(ga, torch.float32, "g_albedo", (N, 3))
    gr = _need(gr, torch.float32, "g_rough", (N,))
    gm = _need(gm, torch.float32, "g_metal", (N,))
    grad_loss = _need(grad_loss, torch.float64, "grad_loss", (1,))
    check(lib().fipt_render_grad_scale(N, _ptr(grad_loss), _ptr(ga), _ptr(gr), _ptr(gm), _stream(stream)))
    return ga, gr, gm


class FactorizedRender(torch.autograd.Function):
    """Tone-mapped factorized-render loss (Eq. 5, 8, 14) with the library's
    hand-written backward for per-point albedo, roughness and metallic.
    When a gradient is needed the forward computes it too (one pass over
    the inputs) and the backward only scales it by the upstream gradient;
    a second backward through the same graph recomputes it."""

    @staticmethod
    def forward(ctx, albedo, rough, metal, Ld, Ls0, Ls1, Lgt, mask, sigma_grid):
        albedo, rough, metal = albedo.contiguous(), rough.contiguous(), metal.contiguous()
        ctx.grads = None
        if any(ctx.needs_input_grad[:3]):
            _, loss, ctx.grads = render_fwd_grad(Ld, Ls0, Ls1, sigma_grid, albedo, rough, metal, Lgt, mask)
        else:
            _, loss = render_fwd(Ld, Ls0, Ls1, sigma_grid, albedo, rough, metal, Lgt, mask)
        ctx.save_for_backward(albedo, rough, metal, Ld, Ls0, Ls1, Lgt,
                              mask if mask is not None else torch.empty(0, device=Ld.device))
        ctx.has_mask = mask is not None
        ctx.sigma_grid = list(sigma_grid)
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().to(torch.float64).reshape(1).contiguous()
        if ctx.grads is not None:        # computed by the forward pass; handed out once
            grads, ctx.grads = ctx.grads, None
            ga, gr, gm = render_grad_scale(grads, g)
        else:
            albedo, rough, metal, Ld, Ls0, Ls1, Lgt, mask = ctx.saved_tensors
            ga, gr, gm = render_bwd(Ld, Ls0, Ls1, ctx.sigma_grid, albedo, rough, metal, Lgt,
                                    mask if ctx.has_mask else None, g)
        return ga, gr, gm, None, None, None, None, None, None


def factorized_render_loss(albedo, rough, metal, tables, Lgt, sigma_grid, mask=None):
    Ld, Ls0, Ls1 = tables
    return FactorizedRender.apply(albedo, rough, metal, Ld, Ls0, Ls1, Lgt, mask, sigma_grid)


def tri_error(tri, Lr, Lgt, T, stream=None, tri_stride=1):
    """Per-triangle sum of ||Lr - Lgt||^2 (float64 [T]) and pixel count (int32 [T]).

    ``tri`` is an int32 tensor of pixel triangle ids, or a [P,10] query tensor
    (its triangle field is read in place, tri_stride = 10)."""
    if tri.dtype == torch.float32 and tri.dim() == 2 and tri.shape[1] == 10:
        tri = _queries(tri, "tri")
        P, tri_stride = tri.shape[0], 10
        tri = tri[:, 9:10]
    else:
        P = tri.shape[0]
        tri = _need(tri, torch.int32, "tri", (P,))
        tri_stride = 1
    Lr = _need(Lr, torch.float32, "Lr", (P, 3))
    Lgt = _need(Lgt, torch.float32, "Lgt", (P, 3))
    nbytes = ctypes.c_size_t()
    check(lib().fipt_tri_error_workspace_size(P, int(T), ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, tri.device)
    err = torch.empty(int(T), dtype=torch.float64, device=tri.device)
    cnt = torch.empty(int(T), dtype=torch.int32, device=tri.device)
    check(lib().fipt_tri_error(_ptr(tri), int(tri_stride), _ptr(Lr), _ptr(Lgt), P, int(T), _ptr(err),
                               _ptr(cnt),
                               _ptr(ws), nbytes.value, _stream(stream)))
    return err, cnt


def emitter_classify(alpha, n_per_tri=100, threshold=0.01, stream=None):
    """Sec. 4.4: a triangle is an emitter when the mean of its n_per_tri mask
    values (alpha, f32 [T * n_per_tri], triangle-major) exceeds threshold.
    Returns (is_emitter u8 [T], mean f64 [T])."""
    alpha = _dev(alpha, torch.float32, "alpha").reshape(-1)
    n = int(n_per_tri)
    if alpha.numel() % n:
        raise ValueError("alpha has %d values, not a multiple of n_per_tri=%d" % (alpha.numel(), n))
    T = alpha.numel() // n
    flag = torch.empty(T, dtype=torch.uint8, device=alpha.device)
    mean = torch.empty(T, dtype=torch.float64, device=alpha.device)
    check(lib().fipt_emitter_classify(_ptr(alpha), T, n, float(threshold), _ptr(mean), _ptr(flag),
                                      _stream(stream)))
    return flag, mean


def emitter_radiance(tri, rgb, is_emitter, stream=None, tri_stride=1):
    """Eq. 12 with zero reflectance at emitters: per-channel (lower) median of
    the radiance rgb [P,3] of the pixels whose first hit is each emitter
    triangle.  ``tri`` as in :func:`tri_error`.  Returns (Le f32 [T,3],
    count i32 [T])."""
    if tri.dtype == torch.float32 and tri.dim() == 2 and tri.shape[1] == 10:
        P, tri_stride = tri.shape[0], 10
        tri = tri[:, 9:10]
    else:
        P = tri.shape[0]
    rgb = _dev(rgb, torch.float32, "rgb")
    is_emitter = _dev(is_emitter, torch.uint8, "is_emitter")
    T = is_emitter.shape[0]
    nbytes = ctypes.c_size_t()
    check(lib().fipt_emitter_radiance_workspace_size(P, T, ctypes.byref(nbytes)))
    _b, ws = _workspace(nbytes.value, rgb.device)
    Le = torch.empty((T, 3), dtype=torch.float32, device=rgb.device)
    cnt = torch.empty(T, dtype=torch.int32, device=rgb.device)
    check(lib().fipt_emitter_radiance(_ptr(tri), int(tri_stride), _ptr(rgb), P, _ptr(is_emitter), T,
                                      _ptr(Le), _ptr(cnt), _ptr(ws), nbytes.value, _stream(stream)))
    return Le, cnt


def extract_emitters(scene: Scene, alpha_fn, pixel_tri, pixel_rgb, n_per_tri=100, threshold=0.01,
                     seed=0, set_emission=True, stream=None):
    """The emitter-extraction step end to end (Sec. 4.4): sample every
    triangle, read the mask field ``alpha_fn(points [M,3]) -> [M]`` there,
    classify, take L_e in closed form from the pixels, and (by default)
    install it as the scene's emission.  Returns (is_emitter, Le, count)."""
    x = scene.emitter_points(n_per_tri, seed=seed, stream=stream)
    alpha = alpha_fn(x).to(torch.float32).reshape(-1)
    flag, _ = emitter_classify(alpha, n_per_tri, threshold, stream=stream)
    Le, cnt = emitter_radiance(pixel_tri, pixel_rgb, flag, stream=stream)
    if set_emission:
        scene.set_emission(Le, stream=stream)
    return flag, Le, cnt


def philox(ctr, key, stream=None):
    """Device Philox4x32-10: ctr [n,4], key [n,2] (int32 tensors holding u32 bits)."""
    n = ctr.shape[0]
    ctr = _need(ctr, torch.int32, "ctr", (n, 4))
    key = _need(key, torch.int32, "key", (n, 2))
    out = torch.empty((n, 4), dtype=torch.int32, device=ctr.device)
    check(lib().fipt_debug_philox(_ptr(ctr), _ptr(key), n, _ptr(out), _stream(stream)))
    return out


class Server:
    """Continuous-batching request loop over resident scenes (fipt_server_*).

    Host inputs should be pinned CPU tensors so copies overlap compute; the
    server allocates pinned host outputs per request."""

    BAKE, RENDER = 0, 1

    def __init__(self, hbm_budget: int, max_batch_rays: int = 1 << 26, chunk_points: int = 16384,
                 ctx: Context | None = None):
        self.ctx = ctx or context()
        h = ctypes.c_void_p()
        check(lib().fipt_server_create(self.ctx.handle, int(hbm_budget), int(max_batch_rays),
                                       int(chunk_points), ctypes.byref(h)))
        self.handle = h
        self._keep = {}
        self._scenes = []
        self._tables = []

    def add_scene(self, scene: "Scene") -> int:
        i = ctypes.c_int32()
        check(lib().fipt_server_add_scene(self.handle, scene.handle, ctypes.byref(i)))
        self._scenes.append(scene)
        return i.value

    def add_table(self, Ld, Ls0, Ls1, sigma_grid) -> int:
        g, K = _grid(sigma_grid)
        i = ctypes.c_int32()
        check(lib().fipt_server_add_table(self.handle, _ptr(Ld), _ptr(Ls0), _ptr(Ls1), Ld.shape[0], K,
                                          g, ctypes.byref(i)))
        self._tables.append((Ld, Ls0, Ls1))
        return i.value

    def _submit(self, req, keep):
        t = ctypes.c_uint64()
        check(lib().fipt_server_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def submit_bake(self, scene_id, queries, sigma, spp_diffuse, spp_specular=None, seed=0,
                    request_id=0):
        """queries: CPU float32 [n,10] (pinned for overlap).  Returns a ticket."""
        n, K = queries.shape[0], len(sigma)
        q = _host(queries, torch.float32, "queries", (n, 10))
        out = {"Ld": torch.empty((n, 3), dtype=torch.float32, pin_memory=True),
               "Ls0": torch.empty((n, K, 3), dtype=torch.float32, pin_memory=True),
               "Ls1": torch.empty((n, K, 3), dtype=torch.float32, pin_memory=True)}
        r = Request()
        r.kind, r.target, r.n, r.first = self.BAKE, int(scene_id), n, 0
        r.queries = q.data_ptr()
        r.params = bake_params(sigma, spp_diffuse, spp_specular, seed, request_id)
        r.Ld, r.Ls0, r.Ls1 = out["Ld"].data_ptr(), out["Ls0"].data_ptr(), out["Ls1"].data_ptr()
        return self._submit(r, {"in": q, "out": out})

    def submit_render(self, table_id, first, albedo, rough, metal, Lgt):
        """Render fwd/bwd over table rows [first, first+n); host tensors in."""
        n = albedo.shape[0]
        ins = [_host(albedo, torch.float32, "albedo", (n, 3)), _host(rough, torch.float32, "rough", (n,)),
               _host(metal, torch.float32, "metal", (n,)), _host(Lgt, torch.float32, "Lgt", (n, 3))]
        out = {"Lr": torch.empty((n, 3), dtype=torch.float32, pin_memory=True),
               "loss": torch.zeros(1, dtype=torch.float64, pin_memory=True),
               "g_albedo": torch.empty((n, 3), dtype=torch.float32, pin_memory=True),
               "g_rough": torch.empty(n, dtype=torch.float32, pin_memory=True),
               "g_metal": torch.empty(n, dtype=torch.float32, pin_memory=True)}
        r = Request()
        r.kind, r.target, r.n, r.first = self.RENDER, int(table_id), n, int(first)
        r.albedo, r.rough, r.metal, r.Lgt = [x.data_ptr() for x in ins]
        r.Lr, r.loss = out["Lr"].data_ptr(), out["loss"].data_ptr()
        r.g_albedo, r.g_rough, r.g_metal = (out["g_albedo"].data_ptr(), out["g_rough"].data_ptr(),
                                            out["g_metal"].data_ptr())
        return self._submit(r, {"in": ins, "out": out})

    def poll(self, ticket):
        done = ctypes.c_int32()
        st = ctypes.c_int()
        check(lib().fipt_server_poll(self.handle, int(ticket), ctypes.byref(done), ctypes.byref(st)))
        return bool(done.value), st.value

    def wait(self, ticket, timeout_s: float = 600.0) -> int:
        """Blocks until the request is done; returns its status (0 = ok)."""
        st = ctypes.c_int()
        check(lib().fipt_server_wait(self.handle, int(ticket), int(timeout_s * 1e6), ctypes.byref(st)))
        return st.value

    def result(self, ticket):
        return self._keep[ticket]["out"]

    def times(self, ticket):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().fipt_server_times(self.handle, int(ticket), ctypes.byref(a), ctypes.byref(b),
                                      ctypes.byref(c)))
        return a.value, b.value, c.value

    def release(self, ticket):
        check(lib().fipt_server_release(self.handle, int(ticket)))
        self._keep.pop(ticket, None)

    def inject_launch_failure(self, after_launches: int = 0):
        """Test hook: the device submission after the next ``after_launches``
        ones fails (FIPT_ERR_CUDA) on the host, as a failed launch would."""
        check(lib().fipt_server_inject_launch_failure(self.handle, int(after_launches)))

    def inject_copy_failure(self, after_steps: int = 0):
        """Test hook: after ``after_steps`` more request copy steps (a
        request's inputs at admission, its outputs at completion), the next
        one is refused on the host as a failed copy call would be; that
        request ends with FIPT_ERR_CUDA and the server goes on."""
        check(lib().fipt_server_inject_copy_failure(self.handle, int(after_steps)))

    def stats(self):
        s = ServerStats()
        check(lib().fipt_server_get_stats(self.handle, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().fipt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
