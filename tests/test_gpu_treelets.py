"""Treelet restructuring of the scene tree (fipt_scene_optimize).

The closest hit is the (t, triangle id) minimum over the triangles a ray
meets, whatever the tree; only where float32 leaves several triangles
within a few ulps of that minimum (a ray along a shared edge, grazing a
face) can the visit order, through the culling bound, pick another of
them -- hits the oracle reports as equally correct.  So a restructured
tree must be a valid binary tree over the same leaves with exact union
boxes, walks on it must visit fewer nodes, its bake must meet the oracle's
bounds, and it may differ from the radix tree's only on a few points.
"""
import numpy as np
import pytest
import torch

from workloads import building_floor, cornell_box, procedural_room, surface_queries

pytestmark = pytest.mark.gpu
SIGMA = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_tree(ex, T, tri_box):
    """Every leaf once, every internal node but the root once, each node's
    box the union of its children's boxes, every leaf reachable from the
    root (vectorised: the floor's tree has 2,045,463 internal nodes)."""
    child, box = ex["child"], ex["box"]
    n = T - 1
    c = child.reshape(-1)
    seen_leaf = np.bincount(~c[c < 0], minlength=T)
    seen_node = np.bincount(c[c >= 0], minlength=n)
    assert len(seen_leaf) == T and len(seen_node) == n
    assert (seen_leaf == 1).all()
    assert seen_node[0] == 0 and (seen_node[1:] == 1).all()
    cb = np.where(child[..., None] < 0, tri_box[np.where(child < 0, ~child, 0)], box[np.where(child >= 0, child, 0)])
    lo = np.minimum(cb[:, 0, :3], cb[:, 1, :3])
    hi = np.maximum(cb[:, 0, 3:], cb[:, 1, 3:])
    assert np.array_equal(np.concatenate([lo, hi], 1), box)
    # reachable from the root, level by level: a walk counts every leaf
    frontier, leaves, levels = np.array([0]), 0, 0
    while frontier.size:
        ch = child[frontier].reshape(-1)
        leaves += int((ch < 0).sum())
        frontier = ch[ch >= 0]
        levels += 1
        assert levels <= n + 1
    assert leaves == T


@pytest.mark.parametrize("mesh", ["cornell", "room", "floor", "dups"])
def test_restructured_tree_is_valid_and_deterministic(fipt, mesh):
    if mesh == "cornell":
        m = cornell_box()
        V, Fi = m.V, m.F
    elif mesh in ("room", "floor"):
        m = procedural_room(1) if mesh == "room" else building_floor(5)
        V, Fi = m.V, m.F
    else:                                    # many triangles with the same centre
        rng = np.random.default_rng(3)
        pts = rng.integers(0, 4, (600, 3)).astype(np.float32)
        V = np.repeat(pts, 3, axis=0) + rng.uniform(0, 0.01, (1800, 3)).astype(np.float32)
        Fi = np.arange(1800, dtype=np.int32).reshape(600, 3)
    T = len(Fi)
    z = cu(np.zeros((T, 3), np.float32))
    exs = []
    for _ in range(2):
        sc = fipt.Scene(cu(V), cu(Fi), z, z, optimize=3)
        exs.append({k: v.cpu().numpy() for k, v in sc.export().items()})
    fipt.context().sync_status()
    assert "range" not in exs[0]
    for k in exs[0]:
        assert np.array_equal(exs[0][k], exs[1][k])          # deterministic
    order = exs[0]["order"]
    tv = V[Fi[order]]
    tri_box = np.concatenate([tv.min(1), tv.max(1)], 1).astype(np.float32)
    check_tree(exs[0], T, tri_box)
    plain = fipt.Scene(cu(V), cu(Fi), z, z, optimize=0)
    ex0 = {k: v.cpu().numpy() for k, v in plain.export().items()}
    assert np.array_equal(ex0["box"][0], exs[0]["box"][0])   # the root box is the scene's
    if mesh != "cornell":
        assert not np.array_equal(ex0["child"], exs[0]["child"])


@pytest.mark.parametrize("mesh,N,spp", [("room", 4000, 16), ("floor", 8192, 8)])
def test_bake_on_restructured_tree(fipt, mesh, N, spp):
    import oracle as O
    from parity import ETA_BAKE, bake_flat, check_bake
    m = procedural_room(1) if mesh == "room" else building_floor(5)
    q = surface_queries(m, N, seed=7)
    out, stats = [], []
    for passes in (0, 1, 3):
        sc = fipt.Scene.from_mesh(m, optimize=passes)
        qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
        st = torch.zeros(4, dtype=torch.int64, device="cuda")
        out.append(bake_flat(*[x.cpu().numpy() for x in fipt.bake(sc, qt, SIGMA, spp, spp, seed=3, stats=st)]))
        stats.append(st.cpu().tolist())
        fipt.context().sync_status()
    for o in out[1:]:
        assert (o != out[0]).any(1).mean() < 0.01           # near-ties only
    rays = stats[0][0]
    nodes = [s_[1] / rays for s_ in stats]
    print("nodes per ray by passes 0, 1, 3:", nodes, "deepest stack:", [s_[3] for s_ in stats])
    assert nodes[1] < nodes[0] and nodes[2] <= nodes[1] * 1.01
    assert max(s_[3] for s_ in stats) <= 32
    if mesh == "room":
        ora = O.OracleScene.from_mesh(m).bake(q, SIGMA, spp, spp, seed=3, eta=ETA_BAKE)
        print(check_bake(out[2], ora))


def test_trace_and_refine_on_restructured_tree(fipt):
    m = procedural_room(1)
    rng = np.random.default_rng(5)
    P = 200000
    o = (m.V.min(0) + rng.uniform(0.05, 0.95, (P, 3)) * (m.V.max(0) - m.V.min(0))).astype(np.float32)
    d = rng.normal(size=(P, 3)).astype(np.float32)
    T = m.T
    a = rng.uniform(0, 1, (T, 3)).astype(np.float32)
    r = rng.uniform(0.02, 1.0, T).astype(np.float32)
    mt = rng.uniform(0, 1, T).astype(np.float32)
    q = surface_queries(m, 2000, seed=9)
    res = []
    for passes in (0, 2):
        sc = fipt.Scene.from_mesh(m, optimize=passes)
        sc.set_materials(cu(a), cu(r), cu(mt))
        hits = [x.cpu().numpy() for x in sc.trace(cu(o), cu(d))]
        qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
        ref = [x.cpu().numpy().reshape(2000, -1) for x in fipt.bake_refine(sc, qt, SIGMA, 8, 8, seed=2)]
        fipt.context().sync_status()
        res.append((hits, np.concatenate(ref, 1)))
    (h0, r0), (h1, r1) = res
    assert (h0[0] != h1[0]).mean() < 1e-4                    # rays from inside the room
    assert (r0 != r1).any(1).mean() < 0.02


@pytest.mark.parametrize("case", ["T3", "T4", "T9", "identical", "planar"])
def test_restructuring_edge_cases(fipt, case):
    """The smallest trees a treelet can reshape, 500 copies of one triangle
    (every box the same: no topology is cheaper, nothing is rewritten) and a
    planar grid (boxes flat in one axis): the tree stays valid and closest
    hits stay those of the radix tree."""
    rng = np.random.default_rng(17)
    if case.startswith("T"):
        T = int(case[1:])
        V = rng.uniform(0, 1, (3 * T, 3)).astype(np.float32)
        Fi = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    elif case == "identical":
        T = 500
        V = np.tile(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), (T, 1))
        Fi = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    else:
        n = 40
        g = np.stack(np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij"), -1).reshape(-1, 2)
        V = np.concatenate([g, np.zeros((len(g), 1))], 1).astype(np.float32)
        idx = lambda i, j: i * (n + 1) + j
        Fi = np.array([[idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)] for i in range(n) for j in range(n)]
                      + [[idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)] for i in range(n) for j in range(n)],
                      np.int32)
        T = len(Fi)
    z = cu(np.zeros((T, 3), np.float32))
    # no relayout where the test asks that restructuring rewrote nothing
    opt = fipt.Scene(cu(V), cu(Fi), z, z, optimize=3, relayout=(case != "identical"))
    plain = fipt.Scene(cu(V), cu(Fi), z, z, optimize=0)
    ex = {k: v.cpu().numpy() for k, v in opt.export().items()}
    ex0 = {k: v.cpu().numpy() for k, v in plain.export().items()}
    tv = V[Fi[ex["order"]]]
    check_tree(ex, T, np.concatenate([tv.min(1), tv.max(1)], 1).astype(np.float32))
    if case == "identical":
        assert np.array_equal(ex["child"], ex0["child"])
    P = 20000
    lo, hi = V.min(0) - 0.5, V.max(0) + 0.5
    o = (lo + rng.uniform(0, 1, (P, 3)) * (hi - lo)).astype(np.float32)
    d = rng.normal(size=(P, 3)).astype(np.float32)
    a = [x.cpu().numpy() for x in opt.trace(cu(o), cu(d))]
    b = [x.cpu().numpy() for x in plain.trace(cu(o), cu(d))]
    fipt.context().sync_status()
    assert np.array_equal(a[0] >= 0, b[0] >= 0)        # a hit exists or not, whatever the tree
    assert (a[0] != b[0]).mean() < 1e-3


def test_relayout_is_depth_first_and_changes_no_result(fipt):
    """fipt_scene_relayout renumbers the internal nodes depth-first (a node's
    first internal child is the next record) without touching the topology:
    the same boxes, the same walks (identical node, triangle and stack
    counts) and bit-identical bakes."""
    m = procedural_room(1)
    T = m.T
    q = surface_queries(m, 20000, seed=13)
    res = []
    for rl in (False, True):
        sc = fipt.Scene.from_mesh(m, optimize=2, relayout=rl)
        ex = {k: v.cpu().numpy() for k, v in sc.export().items()}
        qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
        st = torch.zeros(4, dtype=torch.int64, device="cuda")
        out = [x.cpu() for x in fipt.bake(sc, qt, SIGMA, 16, 16, seed=4, stats=st)]
        fipt.context().sync_status()
        res.append((ex, out, st.cpu().tolist()))
    (ex0, out0, st0), (ex1, out1, st1) = res
    ch = ex1["child"]
    first = np.nonzero(ch[:, 0] >= 0)[0]
    assert np.array_equal(ch[first, 0], first + 1)
    tv = m.V[m.F[ex1["order"]]]
    check_tree(ex1, T, np.concatenate([tv.min(1), tv.max(1)], 1).astype(np.float32))
    key = lambda b: b[np.lexsort(b.T[::-1])]
    assert np.array_equal(key(ex0["box"]), key(ex1["box"]))
    assert st0 == st1
    for x, y in zip(out0, out1):
        assert torch.equal(x, y)
