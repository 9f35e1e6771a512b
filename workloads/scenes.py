"""Procedural scenes, query points, cameras and material parameters.

Every generator is a pure function of its arguments and seed (numpy PCG64),
and returns float32 / int32 arrays in the layouts the C-ABI takes:

* ``Mesh.V``      [nV, 3] float32 vertex positions (metres)
* ``Mesh.F``      [T, 3]  int32 vertex indices; the winding of every triangle
  makes (v1 - v0) x (v2 - v0) point to the side the triangle is seen from
  (into the room for shells, outwards for boxes and spheres, downwards for
  ceiling emitters)
* ``Mesh.Le``     [T, 3]  float32 view-independent emission (Sec. 3)
* ``Mesh.cache``  [T, 3]  float32 per-triangle diffuse radiance cache L'
  (the stand-in for the voxel grid of Sec. 4.2); zero on emitters so that
  emission + cache never counts a triangle twice

Scene recipes (sizes quoted are what the functions produce):

* ``cornell_box()``: unit-cube room with the z=0 face open (10 wall
  triangles), two axis-aligned boxes (24), one 0.3 x 0.3 ceiling emitter
  quad at y=0.999 of radiance (17, 12, 4) (2) -> T = 36; cache 0.5.
* ``procedural_room(seed=1)``: 4 x 6 x 3 m shell on a 0.1 m grid (21,600),
  60 boxes with sides U[0.2, 1.2] m on the floor (720), 30 level-4
  icospheres of radius U[0.1, 0.4] m (153,600), 3 ceiling emitters with
  sides U[0.5, 1.2] m and grey radiance log-U[5, 50] (6) -> T = 175,926;
  cache U[0, 1]^3.
* ``building_floor(seed=5, rooms=4)``: four 5 x 6 x 3 m rooms side by side
  along x with 0.2 m between shells, shells on a 0.05 m grid (403,200),
  80 boxes (3,840), 20 level-5 icospheres (1,638,400) and 3 emitters (24)
  per room -> T = 2,045,464.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    V: np.ndarray
    F: np.ndarray
    Le: np.ndarray
    cache: np.ndarray
    emitter: np.ndarray          # [T] bool
    sample_ok: np.ndarray        # [T] bool: query points may be drawn here
    floor: np.ndarray            # [T] bool: triangle lies on a room floor
    footprints: np.ndarray       # [nb, 4] (x0, x1, z0, z1) floor areas under boxes
    rooms: list = field(default_factory=list)   # [(lo[3], hi[3])] room interiors
    spheres: np.ndarray = None   # [ns, 4] centre xyz, radius
    boxes: np.ndarray = None     # [nb, 6] lo xyz, hi xyz
    name: str = ""

    @property
    def T(self) -> int:
        return int(self.F.shape[0])


class _Builder:
    """Accumulates triangle soups with a per-triangle tag."""

    NORMAL, EMITTER, HIDDEN = 0, 1, 2

    def __init__(self):
        self.V, self.F, self.tag, self.floor = [], [], [], []
        self.nv = 0

    def add(self, V, F, tag, floor=False):
        V = np.asarray(V, np.float64)
        F = np.asarray(F, np.int64) + self.nv
        self.V.append(V)
        self.F.append(F)
        self.tag.append(np.full(len(F), tag, np.int8))
        self.floor.append(np.full(len(F), floor, bool))
        self.nv += len(V)

    def grid(self, origin, du, dv, nu, nv, normal, tag=0, floor=False):
        """Planar rectangle origin + s*du + t*dv split into nu x nv cells,
        two triangles per cell, wound so that the face normal is ``normal``."""
        origin, du, dv = (np.asarray(a, np.float64) for a in (origin, du, dv))
        iu = np.arange(nu + 1, dtype=np.float64) / nu
        iv = np.arange(nv + 1, dtype=np.float64) / nv
        S, Tt = np.meshgrid(iu, iv, indexing="ij")
        V = origin + S[..., None] * du + Tt[..., None] * dv
        V = V.reshape(-1, 3)
        idx = np.arange((nu + 1) * (nv + 1)).reshape(nu + 1, nv + 1)
        a = idx[:-1, :-1].ravel()
        b = idx[1:, :-1].ravel()
        c = idx[1:, 1:].ravel()
        d = idx[:-1, 1:].ravel()
        if np.dot(np.cross(du, dv), normal) > 0:
            F = np.concatenate([np.stack([a, b, c], 1), np.stack([a, c, d], 1)])
        else:
            F = np.concatenate([np.stack([a, c, b], 1), np.stack([a, d, c], 1)])
        self.add(V, F, tag, floor)

    def box(self, lo, hi, hidden_bottom=True):
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        ex = hi - lo
        X, Y, Z = np.eye(3)
        self.grid(lo, [ex[0], 0, 0], [0, 0, ex[2]], 1, 1, -Y,
                  self.HIDDEN if hidden_bottom else self.NORMAL)      # bottom
        self.grid([lo[0], hi[1], lo[2]], [ex[0], 0, 0], [0, 0, ex[2]], 1, 1, Y)  # top
        self.grid(lo, [0, ex[1], 0], [0, 0, ex[2]], 1, 1, -X)          # x-
        self.grid([hi[0], lo[1], lo[2]], [0, ex[1], 0], [0, 0, ex[2]], 1, 1, X)  # x+
        self.grid(lo, [ex[0], 0, 0], [0, ex[1], 0], 1, 1, -Z)          # z-
        self.grid([lo[0], lo[1], hi[2]], [ex[0], 0, 0], [0, ex[1], 0], 1, 1, Z)  # z+

    def shell(self, lo, hi, step, open_front=False):
        """Closed axis-aligned room seen from inside, on a square grid."""
        lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
        ex = hi - lo
        n = [int(round(e / step)) for e in ex]
        X, Y, Z = np.eye(3)
        self.grid(lo, [ex[0], 0, 0], [0, 0, ex[2]], n[0], n[2], Y, floor=True)          # floor
        self.grid([lo[0], hi[1], lo[2]], [ex[0], 0, 0], [0, 0, ex[2]], n[0], n[2], -Y)  # ceiling
        self.grid(lo, [0, ex[1], 0], [0, 0, ex[2]], n[1], n[2], X)                      # x = lo
        self.grid([hi[0], lo[1], lo[2]], [0, ex[1], 0], [0, 0, ex[2]], n[1], n[2], -X)  # x = hi
        self.grid([lo[0], lo[1], hi[2]], [ex[0], 0, 0], [0, ex[1], 0], n[0], n[1], -Z)  # z = hi
        if not open_front:
            self.grid(lo, [ex[0], 0, 0], [0, ex[1], 0], n[0], n[1], Z)                  # z = lo

    def ceiling_emitter(self, x0, z0, sx, sz, y):
        self.grid([x0, y, z0], [sx, 0, 0], [0, 0, sz], 1, 1, [0, -1, 0], self.EMITTER)

    def sphere(self, unit_V, unit_F, centre, radius):
        self.add(np.asarray(centre) + radius * unit_V, unit_F, self.NORMAL)

    def finish(self):
        V = np.concatenate(self.V).astype(np.float32)
        F = np.concatenate(self.F).astype(np.int32)
        tag = np.concatenate(self.tag)
        floor = np.concatenate(self.floor)
        return V, F, tag, floor


def _icosphere(level: int):
    """Unit icosphere: icosahedron split ``level`` times, outward winding."""
    p = (1.0 + 5.0 ** 0.5) / 2.0
    V = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
         (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
         (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    V = [np.array(v, np.float64) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        mid = {}

        def m(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                v = V[a] + V[b]
                V.append(v / np.linalg.norm(v))
                mid[key] = len(V) - 1
            return mid[key]

        nF = []
        for a, b, c in F:
            ab, bc, ca = m(a, b), m(b, c), m(c, a)
            nF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nF
    V = np.array(V)
    F = np.array(F, np.int64)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = (n * V[F].mean(1)).sum(1) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


_ICO_CACHE: dict = {}


def _ico(level):
    if level not in _ICO_CACHE:
        _ICO_CACHE[level] = _icosphere(level)
    return _ICO_CACHE[level]


def _mesh(b: _Builder, Le_of_emitter, cache, name, footprints, rooms,
          spheres, boxes) -> Mesh:
    V, F, tag, floor = b.finish()
    T = len(F)
    emitter = tag == _Builder.EMITTER
    Le = np.zeros((T, 3), np.float32)
    Le[emitter] = Le_of_emitter
    cache = np.asarray(cache, np.float32)
    if cache.ndim == 1:
        cache = np.broadcast_to(cache, (T, 3)).copy()
    cache[emitter] = 0.0
    sample_ok = tag == _Builder.NORMAL
    return Mesh(V, F, Le, cache, emitter, sample_ok, floor,
                np.asarray(footprints, np.float64).reshape(-1, 4), rooms,
                np.asarray(spheres, np.float64).reshape(-1, 4),
                np.asarray(boxes, np.float64).reshape(-1, 6), name)


def cornell_box(closed: bool = False, with_boxes: bool = True,
                furnace_radiance: float | None = None,
                cache_value: float = 0.5) -> Mesh:
    """The 36-triangle Cornell box.

    ``closed`` adds the z=0 wall (12 wall triangles) so that every ray from
    inside hits something; ``furnace_radiance`` turns the emitter off and sets
    the cache of every triangle (emitter included) to that value, which makes
    the closed box a uniform-radiance enclosure.
    """
    b = _Builder()
    b.shell([0, 0, 0], [1, 1, 1], 1.0, open_front=not closed)
    boxes, fps = [], []
    if with_boxes:
        for lo, hi in (([0.55, 0.0, 0.15], [0.85, 0.30, 0.45]),
                       ([0.15, 0.0, 0.50], [0.45, 0.60, 0.80])):
            b.box(lo, hi)
            boxes.append(lo + hi)
            fps.append([lo[0], hi[0], lo[2], hi[2]])
    b.ceiling_emitter(0.35, 0.35, 0.3, 0.3, 0.999)
    if furnace_radiance is None:
        m = _mesh(b, [17.0, 12.0, 4.0], [cache_value] * 3, "cornell",
                  fps, [([0, 0, 0], [1, 1, 1])], [], boxes)
    else:
        m = _mesh(b, [0.0, 0.0, 0.0], [furnace_radiance] * 3, "furnace",
                  fps, [([0, 0, 0], [1, 1, 1])], [], boxes)
        m.cache[:] = furnace_radiance
    return m


def _furnish_room(b, rng, lo, hi, n_boxes, n_spheres, ico_level, n_emit,
                  boxes, fps, spheres):
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    uV, uF = _ico(ico_level)
    for _ in range(n_boxes):
        s = rng.uniform(0.2, 1.2, 3)
        x0 = rng.uniform(lo[0] + 0.05, hi[0] - s[0] - 0.05)
        z0 = rng.uniform(lo[2] + 0.05, hi[2] - s[2] - 0.05)
        blo = np.array([x0, lo[1], z0])
        bhi = blo + s
        b.box(blo, bhi)
        boxes.append(np.concatenate([blo, bhi]))
        fps.append([blo[0], bhi[0], blo[2], bhi[2]])
    for _ in range(n_spheres):
        r = rng.uniform(0.1, 0.4)
        c = rng.uniform(lo + r, hi - r)
        b.sphere(uV, uF, c, r)
        spheres.append([c[0], c[1], c[2], r])
    le = []
    for _ in range(n_emit):
        sx, sz = rng.uniform(0.5, 1.2, 2)
        x0 = rng.uniform(lo[0] + 0.1, hi[0] - sx - 0.1)
        z0 = rng.uniform(lo[2] + 0.1, hi[2] - sz - 0.1)
        b.ceiling_emitter(x0, z0, sx, sz, hi[1] - 0.01)
        le.append(np.exp(rng.uniform(np.log(5.0), np.log(50.0))))
    return le


def procedural_room(seed: int = 1) -> Mesh:
    """The ~176k-triangle indoor room (shell, 60 boxes, 30 spheres, 3 lights)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    lo, hi = [0.0, 0.0, 0.0], [4.0, 3.0, 6.0]
    b.shell(lo, hi, 0.1)
    boxes, fps, spheres = [], [], []
    le = _furnish_room(b, rng, lo, hi, 60, 30, 4, 3, boxes, fps, spheres)
    V, F, tag, floor = b.finish()
    T = len(F)
    emitter = tag == _Builder.EMITTER
    Le = np.zeros((T, 3), np.float32)
    Le[emitter] = np.repeat(np.asarray(le, np.float32), 2)[:, None]
    cache = rng.uniform(0.0, 1.0, (T, 3)).astype(np.float32)
    cache[emitter] = 0.0
    return Mesh(V, F, Le, cache, emitter, tag == _Builder.NORMAL, floor,
                np.asarray(fps).reshape(-1, 4), [(np.array(lo), np.array(hi))],
                np.asarray(spheres).reshape(-1, 4), np.asarray(boxes).reshape(-1, 6),
                "room")


def building_floor(seed: int = 5, rooms: int = 4, step: float = 0.05,
                   boxes_per_room: int = 80, spheres_per_room: int = 20,
                   ico_level: int = 5) -> Mesh:
    """Closed rooms side by side along x (0.2 m between shells)."""
    rng = np.random.default_rng(seed)
    b = _Builder()
    boxes, fps, spheres, le, room_list = [], [], [], [], []
    for r in range(rooms):
        lo = [5.2 * r, 0.0, 0.0]
        hi = [5.2 * r + 5.0, 3.0, 6.0]
        b.shell(lo, hi, step)
        room_list.append((np.array(lo), np.array(hi)))
        le += _furnish_room(b, rng, lo, hi, boxes_per_room, spheres_per_room,
                            ico_level, 3, boxes, fps, spheres)
    V, F, tag, floor = b.finish()
    T = len(F)
    emitter = tag == _Builder.EMITTER
    Le = np.zeros((T, 3), np.float32)
    Le[emitter] = np.repeat(np.asarray(le, np.float32), 2)[:, None]
    cache = rng.uniform(0.0, 1.0, (T, 3)).astype(np.float32)
    cache[emitter] = 0.0
    return Mesh(V, F, Le, cache, emitter, tag == _Builder.NORMAL, floor,
                np.asarray(fps).reshape(-1, 4), room_list,
                np.asarray(spheres).reshape(-1, 4), np.asarray(boxes).reshape(-1, 6),
                "floor%d" % rooms)


def surface_queries(mesh: Mesh, n: int, seed: int = 0, min_cos: float = 0.05,
                    all_triangles: bool = False):
    """Area-uniform query points on the triangles marked ``sample_ok`` (every
    triangle, with no footprint rejection, when ``all_triangles``).

    Returns a dict of float32 arrays ``x`` [n,3], ``n`` [n,3] (unit face normal
    on the visible side), ``wo`` [n,3] (unit viewing direction with
    cosine-weighted density about ``n`` and n.wo >= min_cos) and int32 ``tri``
    [n].  Floor points inside a box footprint are redrawn.
    """
    rng = np.random.default_rng(seed)
    V = mesh.V.astype(np.float64)
    F = mesh.F
    cand = np.arange(mesh.T) if all_triangles else np.nonzero(mesh.sample_ok)[0]
    v0, v1, v2 = V[F[cand, 0]], V[F[cand, 1]], V[F[cand, 2]]
    cr = np.cross(v1 - v0, v2 - v0)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    p = area / area.sum()
    xs, ts = [], []
    need = n
    while need > 0:
        k = cand_idx = rng.choice(len(cand), size=2 * need + 16, p=p)
        u = rng.random(len(k))
        w = rng.random(len(k))
        r1 = np.sqrt(u)
        x = ((1 - r1)[:, None] * v0[k] + (r1 * (1 - w))[:, None] * v1[k]
             + (r1 * w)[:, None] * v2[k])
        ok = np.ones(len(k), bool)
        onfloor = mesh.floor[cand[k]]
        for x0, x1, z0, z1 in ([] if all_triangles else mesh.footprints):
            inside = (x[:, 0] >= x0) & (x[:, 0] <= x1) & (x[:, 2] >= z0) & (x[:, 2] <= z1)
            ok &= ~(onfloor & inside)
        xs.append(x[ok])
        ts.append(cand[cand_idx[ok]])
        need -= int(ok.sum())
    x = np.concatenate(xs)[:n]
    tri = np.concatenate(ts)[:n]
    nrm = np.cross(V[F[tri, 1]] - V[F[tri, 0]], V[F[tri, 2]] - V[F[tri, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    # Viewing directions: a point drawn uniformly in the unit disk lifted to
    # the hemisphere has density proportional to n.wo; redraw below min_cos.
    wo = np.empty_like(nrm)
    todo = np.arange(n)
    while len(todo):
        d = rng.uniform(-1.0, 1.0, (len(todo), 2))
        r2 = (d * d).sum(1)
        z2 = 1.0 - r2
        good = (r2 < 1.0) & (z2 >= min_cos * min_cos)
        sel = todo[good]
        d, z = d[good], np.sqrt(z2[good])
        nn = nrm[sel]
        helper = np.where(np.abs(nn[:, :1]) < 0.9, [[1.0, 0, 0]], [[0, 1.0, 0]])
        e1 = np.cross(nn, helper)
        e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
        e2 = np.cross(nn, e1)
        wo[sel] = d[:, :1] * e1 + d[:, 1:] * e2 + z[:, None] * nn
        todo = todo[~good]
    wo /= np.linalg.norm(wo, axis=1, keepdims=True)
    return {"x": x.astype(np.float32), "n": nrm.astype(np.float32),
            "wo": wo.astype(np.float32), "tri": tri.astype(np.int32)}


def pinhole_views(mesh: Mesh, n_views: int, seed: int = 2,
                  vfov_deg: float = 60.0):
    """Pinhole cameras spread over the mesh's rooms, [n_views, 10] float32.

    Row layout: eye xyz, forward xyz (unit), up xyz (unit, world +y),
    vertical field of view in radians.  Eyes are uniform over the room at a
    height of 1.2-1.8 m, 0.3 m from the walls and clear of boxes and spheres;
    yaw is uniform and pitch U[-20, 20] degrees.  View v is placed in room
    v mod len(mesh.rooms).
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((n_views, 10), np.float64)
    for v in range(n_views):
        lo, hi = mesh.rooms[v % len(mesh.rooms)]
        while True:
            eye = np.array([rng.uniform(lo[0] + 0.3, hi[0] - 0.3),
                            rng.uniform(lo[1] + 1.2, lo[1] + 1.8),
                            rng.uniform(lo[2] + 0.3, hi[2] - 0.3)])
            clear = True
            for cx, cy, cz, r in mesh.spheres:
                if np.linalg.norm(eye - [cx, cy, cz]) < r + 0.05:
                    clear = False
            for bx in mesh.boxes:
                if np.all(eye > bx[:3] - 0.05) and np.all(eye < bx[3:] + 0.05):
                    clear = False
            if clear:
                break
        yaw = rng.uniform(0.0, 2.0 * np.pi)
        pitch = np.deg2rad(rng.uniform(-20.0, 20.0))
        fwd = np.array([np.cos(pitch) * np.sin(yaw), np.sin(pitch),
                        np.cos(pitch) * np.cos(yaw)])
        out[v, 0:3] = eye
        out[v, 3:6] = fwd
        out[v, 6:9] = [0.0, 1.0, 0.0]
        out[v, 9] = np.deg2rad(vfov_deg)
    return out.astype(np.float32)


def material_params(n: int, seed: int = 3):
    """Per-point albedo U[0,1]^3, roughness U[0.02,1], metallic U[0,1]."""
    rng = np.random.default_rng(seed)
    return {"albedo": rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32),
            "rough": rng.uniform(0.02, 1.0, n).astype(np.float32),
            "metal": rng.uniform(0.0, 1.0, n).astype(np.float32)}


def shading_tables(n: int, K: int = 6, seed: int = 7):
    """Synthetic shading tables of the baked layout for render tests:
    Ld [n,3], Ls0 [n,K,3], Ls1 [n,K,3] float32, non-negative, with L_s0
    and L_s1 smooth in the roughness index (radiance-like magnitudes)."""
    rng = np.random.default_rng(seed)
    base = np.exp(rng.uniform(np.log(0.05), np.log(5.0), (n, 1, 3)))
    ramp = np.linspace(1.0, 0.4, K)[None, :, None]
    Ld = (base[:, 0] * rng.uniform(0.5, 1.5, (n, 3))).astype(np.float32)
    Ls0 = (base * ramp * rng.uniform(0.8, 1.2, (n, K, 3))).astype(np.float32)
    Ls1 = (0.1 * base * ramp * rng.uniform(0.8, 1.2, (n, K, 3))).astype(np.float32)
    return Ld, Ls0, Ls1


def emitter_pixels(mesh: Mesh, P: int, seed: int = 0, miss_frac: float = 0.1,
                   emitter_frac: float = 0.3, outlier_frac: float = 0.05):
    """Input pixels for emitter extraction: (tri int32 [P], rgb float32 [P,3]).

    A fraction ``miss_frac`` of pixels hits nothing (tri = -1), a fraction
    ``emitter_frac`` hits an emitter triangle (uniform over them) with
    radiance L_e times a per-channel lognormal factor of median 1 (sigma
    0.2), the rest hit other triangles with radiance U[0, 1]^3.  A fraction
    ``outlier_frac`` of all pixels is scaled by U[3, 10] (highlights)."""
    rng = np.random.default_rng(seed)
    em = np.nonzero(mesh.emitter)[0]
    other = np.nonzero(~mesh.emitter)[0]
    kind = rng.uniform(size=P)
    tri = np.full(P, -1, np.int64)
    on_e = (kind >= miss_frac) & (kind < miss_frac + emitter_frac) & (len(em) > 0)
    on_o = kind >= miss_frac + emitter_frac
    tri[on_e] = em[rng.integers(0, max(len(em), 1), on_e.sum())] if len(em) else -1
    tri[on_o] = other[rng.integers(0, len(other), on_o.sum())]
    rgb = rng.uniform(0.0, 1.0, (P, 3))
    rgb[on_e] = mesh.Le[tri[on_e]] * rng.lognormal(0.0, 0.2, (on_e.sum(), 3))
    out = rng.uniform(size=P) < outlier_frac
    rgb[out] *= rng.uniform(3.0, 10.0, (out.sum(), 1))
    return tri.astype(np.int32), rgb.astype(np.float32)
