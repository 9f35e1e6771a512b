"""Emitter extraction (Sec. 4.4, Eq. 12) on the GPU vs the oracle.

The sample points are float32 on the GPU and FP64 in the oracle: they agree
to float32 rounding of the vertex combination (|x| <= scene size, so within
8 ulp of the scene's largest coordinate).  Classification (FP64 mean in
sample order) and the median (a selection of input values) are exact, so
flags, means, counts and L_e compare bit for bit."""
import numpy as np
import pytest
import torch

import oracle as O
from conftest import read_golden
from workloads import cornell_box, emitter_pixels, procedural_room, surface_queries

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("mesh,n", [("cornell", 100), ("room", 3), ("cornell", 1), ("cornell", 2),
                                    ("cornell", 7), ("cornell", 64), ("cornell", 1000)])
def test_points_match_oracle(fipt, mesh, n):
    m = cornell_box() if mesh == "cornell" else procedural_room(1)
    sc = fipt.Scene.from_mesh(m)
    g = sc.emitter_points(n, seed=11, request_id=2).cpu().numpy().astype(np.float64)
    o = O.OracleScene.from_mesh(m).emitter_points(n, seed=11, request_id=2)
    scale = np.abs(m.V).max()
    assert np.max(np.abs(g - o)) <= 8 * scale * 2.0 ** -24


def test_classify_bit_exact(fipt):
    rng = np.random.default_rng(3)
    T, n = 20000, 100
    alpha = rng.uniform(0, 1, (T, n)).astype(np.float32) ** 8        # most means near 0.1
    alpha[: T // 2] *= np.float32(0.1)                                 # and many near 0.01
    g_flag, g_mean = fipt.emitter_classify(cu(alpha.reshape(-1)), n, 0.01)
    o_flag, o_mean = O.emitter_classify(alpha.reshape(-1), n, 0.01)
    assert np.array_equal(g_mean.cpu().numpy(), o_mean)
    assert np.array_equal(g_flag.cpu().numpy(), o_flag)
    assert 0.05 < o_flag.mean() < 0.95


@pytest.mark.parametrize("n,offset", [(1, 0), (3, 0), (31, 0), (32, 0), (33, 0), (100, 0), (100, 1), (127, 0),
                                      (127, 3), (128, 0), (1000, 0)])
def test_classify_row_kinds_bit_exact(fipt, n, offset):
    """Rows of every kind the mean can meet, at row lengths around the warp
    width: ordinary values, zeros only, two-valued masks, both signs with
    cancellations, values 2^-60 apart, subnormals, infinities and NaNs; the
    mean is the in-order FP64 sum over n on both sides, bit for bit.  Rows
    of up to 127 samples are staged through shared memory and longer ones
    are not; a nonzero offset starts alpha off a 16-byte boundary."""
    rng = np.random.default_rng(n)
    kinds = 9
    T = kinds * 40
    a = np.empty((T, n), np.float32)
    for t in range(T):
        k = t % kinds
        if k == 0:
            r = rng.uniform(0, 1, n)
        elif k == 1:
            r = np.zeros(n)
        elif k == 2:
            r = (rng.uniform(size=n) < 0.3) * 0.05
        elif k == 3:
            r = rng.uniform(-1, 1, n) * 2.0 ** rng.integers(-8, 8, n)
            r[::2] = -np.roll(r, 1)[::2]
        elif k == 4:
            r = rng.uniform(0.5, 1, n) * 2.0 ** rng.integers(-60, 1, n)
        elif k == 5:
            r = rng.uniform(0, 1, n)
            r[rng.integers(0, n)] = 1e-41
        elif k == 6:
            r = rng.uniform(0, 1, n)
            r[rng.integers(0, n)] = np.inf
        elif k == 7:
            r = rng.uniform(0, 1, n)
            r[rng.integers(0, n)] = np.nan
        else:
            r = rng.uniform(0, 0.02, n) * 2.0 ** rng.integers(-20, 0, n)
        a[t] = r
    buf = cu(np.concatenate([np.zeros(offset, np.float32), a.reshape(-1)]))
    g_flag, g_mean = fipt.emitter_classify(buf[offset:], n, 0.01)
    o_flag, o_mean = O.emitter_classify(a.reshape(-1), n, 0.01)
    g_mean = g_mean.cpu().numpy()
    assert np.array_equal(np.isnan(g_mean), np.isnan(o_mean))
    ok = ~np.isnan(o_mean)
    assert np.array_equal(g_mean[ok].view(np.uint64), o_mean[ok].view(np.uint64))
    assert np.array_equal(g_flag.cpu().numpy(), o_flag)


def test_worked_example(fipt):
    rows = read_golden("emitter_extraction_worked_example.txt")
    alpha = np.array([[float(v) for v in r[2:]] for r in rows if r[0] == "alpha"], np.float32)
    pix = [r[1:] for r in rows if r[0] == "pixel"]
    tri = np.array([int(r[0]) for r in pix], np.int32)
    rgb = np.array([[float(v) for v in r[1:]] for r in pix], np.float32)
    want = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "want"])
    flag, _ = fipt.emitter_classify(cu(alpha.reshape(-1)), 4, 0.01)
    assert flag.cpu().numpy().tolist() == want[:, 1].astype(int).tolist()
    Le, cnt = fipt.emitter_radiance(cu(tri), cu(rgb), flag)
    assert cnt.cpu().numpy().tolist() == want[:, 2].astype(int).tolist()
    assert np.array_equal(Le.cpu().numpy(), want[:, 3:6].astype(np.float32))


@pytest.mark.parametrize("P,T,seed", [(0, 5, 1), (1, 1, 2), (777, 3, 3), (100003, 513, 4),
                                      (2000000, 175926, 5)])
def test_radiance_bit_exact(fipt, P, T, seed):
    rng = np.random.default_rng(seed)
    flag = (rng.uniform(size=T) < 0.5).astype(np.uint8)
    tri = rng.integers(-2, T + 2, P).astype(np.int32)                # includes ids out of range
    rgb = (rng.lognormal(0, 1.5, (P, 3)) * rng.choice([1, -1], (P, 3), p=[0.95, 0.05])).astype(np.float32)
    rgb[rng.uniform(size=P) < 0.01] = 0.0
    rgb[rng.uniform(size=P) < 0.01] = -0.0
    rgb[rng.uniform(size=P) < 0.01] = np.inf
    Le, cnt = fipt.emitter_radiance(cu(tri), cu(rgb), cu(flag))
    oLe, ocnt = O.emitter_radiance(tri, rgb, flag)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    g = Le.cpu().numpy()
    assert np.array_equal(g.view(np.uint32), oLe.view(np.uint32))   # signed zeros too


def test_radiance_from_query_records(fipt):
    m = procedural_room(1)
    sc = fipt.Scene.from_mesh(m)
    from workloads import pinhole_views
    cams = cu(pinhole_views(m, 4, seed=3))
    q, valid = sc.camera_queries(cams, 160, 104)
    P = q.shape[0]
    rng = np.random.default_rng(9)
    rgb = rng.uniform(0, 5, (P, 3)).astype(np.float32)
    flag = m.emitter.astype(np.uint8)
    flag[::7] = 1
    Le, cnt = fipt.emitter_radiance(q, cu(rgb), cu(flag))
    tri = q[:, 9].contiguous().view(torch.int32).cpu().numpy()
    oLe, ocnt = O.emitter_radiance(tri, rgb, flag)
    assert np.array_equal(cnt.cpu().numpy(), ocnt)
    assert np.array_equal(Le.cpu().numpy(), oLe)
    assert ocnt.sum() > 1000


def test_set_emission_equals_a_scene_built_with_it(fipt):
    """After set_emission the bake and the refinement (whose MIS samples the
    emitter table) give the bytes of a scene created with that L_e."""
    m = cornell_box()
    T = m.T
    rng = np.random.default_rng(2)
    Le = np.zeros((T, 3), np.float32)
    pick = rng.choice(T, 5, replace=False)
    Le[pick] = rng.uniform(1, 10, (5, 3))
    a = np.full((T, 3), 0.6, np.float32)
    r = np.full(T, 0.3, np.float32)
    r[m.floor] = 0.05
    mt = np.zeros(T, np.float32)
    q = surface_queries(m, 500, seed=3)
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    A = fipt.Scene.from_mesh(m)
    A.set_emission(cu(Le))
    B = fipt.Scene(cu(m.V), cu(m.F), cu(Le), cu(m.cache))
    outs = []
    for sc in (A, B):
        sc.set_materials(cu(a), cu(r), cu(mt))
        outs.append([x.cpu().numpy() for x in fipt.bake(sc, qt, [0.1, 0.5], 16, 8, seed=1)]
                    + [x.cpu().numpy() for x in fipt.bake_refine(sc, qt, [0.1, 0.5], 8, 8, seed=1)])
    for x, y in zip(*outs):
        assert np.array_equal(x, y)
    assert np.abs(outs[0][0]).sum() > 0


def test_extract_emitters_end_to_end(fipt):
    """Mask field = 1 within 0.4 mm of the light's plane (y = 0.999, under
    the ceiling at y = 1) inside its square, 0 elsewhere; pixels from the
    synthetic capture.  The light's triangles are found and their L_e
    recovered; the rest of the scene stays dark."""
    m = cornell_box()
    sc = fipt.Scene(cu(m.V), cu(m.F), cu(np.zeros_like(m.Le)), cu(m.cache))

    def alpha_fn(x):
        on = (((x[:, 1] - 0.999).abs() < 4e-4) & (x[:, 0] > 0.35) & (x[:, 0] < 0.65)
              & (x[:, 2] > 0.35) & (x[:, 2] < 0.65))
        return on.float()

    tri, rgb = emitter_pixels(m, 300000, seed=6)
    flag, Le, cnt = fipt.extract_emitters(sc, alpha_fn, cu(tri), cu(rgb), n_per_tri=100)
    assert np.array_equal(flag.cpu().numpy().astype(bool), m.emitter)
    oLe, ocnt = O.emitter_radiance(tri, rgb, m.emitter.astype(np.uint8))
    assert np.array_equal(Le.cpu().numpy(), oLe)
    assert np.allclose(oLe[m.emitter], m.Le[m.emitter], rtol=0.03)


def test_emitter_detection_sanity_on_the_floor(fipt):
    """The large-scene configuration end to end (Sec. 4.4): first hits of 64
    256x256 views of the 2,045,464-triangle floor, shading tables baked at
    16 spp, targets = the factorized render with true materials plus the
    emission of emitter hits, renders with perturbed materials.  Ranked by
    mean per-pixel error, the top-c triangles (c = emitter triangles that
    some pixel sees) are those emitters (IoU >= 0.9)."""
    from workloads import building_floor, material_params, pinhole_views
    m = building_floor(5)
    sc = fipt.Scene.from_mesh(m)
    qa, valid = sc.camera_queries(cu(pinhole_views(m, 64, seed=2)), 256, 256)
    q, _pix, n = fipt.compact_queries(qa, valid, qa.shape[0])
    q = q[:int(n.item())]
    N = q.shape[0]
    sigma = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
    Ld, Ls0, Ls1 = fipt.bake(sc, q, sigma, 16, 16, seed=4)
    true, est = material_params(N, seed=3), material_params(N, seed=3)
    rng = np.random.default_rng(5)
    est["albedo"] = np.clip(est["albedo"] * rng.uniform(0.9, 1.1, est["albedo"].shape), 0, 1).astype(np.float32)
    est["rough"] = np.clip(est["rough"] + rng.normal(0, 0.02, N), 0.02, 1).astype(np.float32)
    tri = q[:, 9].contiguous().view(torch.int32)
    Lgt = fipt.render_fwd(Ld, Ls0, Ls1, sigma, cu(true["albedo"]), cu(true["rough"]), cu(true["metal"]))[0]
    Lgt = Lgt + cu(m.Le)[tri.long()]
    Lr = fipt.render_fwd(Ld, Ls0, Ls1, sigma, cu(est["albedo"]), cu(est["rough"]), cu(est["metal"]))[0]
    err, cnt = fipt.tri_error(q, Lr, Lgt, m.T)
    fipt.context().sync_status()
    err, cnt = err.cpu().numpy(), cnt.cpu().numpy()
    seen = np.nonzero(m.emitter & (cnt > 0))[0]
    assert len(seen) >= 4
    mean = np.where(cnt > 0, err / np.maximum(cnt, 1), -1.0)
    top = np.argsort(-mean, kind="stable")[:len(seen)]
    iou = len(set(top) & set(seen)) / len(set(top) | set(seen))
    assert iou >= 0.9, (iou, len(seen))
