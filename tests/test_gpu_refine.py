"""GPU stage-3 refinement (Sec. 4.3, Eq. 10, MIS) vs the FP64 oracle on the
same Philox streams.

Multi-bounce paths branch on float decisions (which triangle a ray hits,
which lobe a vertex draws, which emitter triangle an area sample picks,
whether a glossy lobe's D is evaluated a rounding away); for every sample
the oracle returns the range of its value over every decision that the
float32 path's accumulated rounding may flip.  Every GPU sample must lie in
its range widened by 1e-4 (relative to the larger of the oracle's value
and the column's mean), and so must every per-point estimate (the mean of
its samples' ranges).  Where a path's hit points become more uncertain than
1e-4 of the scene (rounding grows by about 1/cos per bounce, so deep glossy
paths lose track of their FP64 twin) the sample's range is [0, inf]; those
samples are compared statistically: their GPU mean equals the oracle's
within four standard errors."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import cornell_box, procedural_room, surface_queries

pytestmark = pytest.mark.gpu
SIGMA = [0.02, 0.25, 1.0]
ETA = 1e-5
REL = 1e-4


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_both(F, m, q, albedo, rough, metal, spp, mis=True, sigma_c=0.6, max_depth=8, seed=3):
    sc = F.Scene.from_mesh(m)
    sc.set_materials(cu(albedo), cu(rough), cu(metal))
    qt = F.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    Ld, Ls0, Ls1, ps = F.bake_refine(sc, qt, SIGMA, spp, spp, sigma_c=sigma_c, max_depth=max_depth,
                                     mis=mis, seed=seed, request_id=1, per_sample=True)
    F.context().sync_status()
    ora = O.OracleScene.from_mesh(m).refine(q, SIGMA, spp, spp, albedo, rough, metal,
                                            sigma_c=sigma_c, max_depth=max_depth, mis=mis,
                                            seed=seed, request_id=1, eta=ETA, per_sample=True,
                                            bounds=True)
    g = {"Ld": Ld.cpu().numpy(), "Ls0": Ls0.cpu().numpy(), "Ls1": Ls1.cpu().numpy(),
         "ps": ps.cpu().numpy().astype(np.float64)}
    return g, ora


def check(g, ora, spp, max_unbounded):
    """Every sample within its range (bounded samples) or statistically
    equal (unbounded ones); every per-point value within the mean of its
    samples' ranges.  Returns (fraction of samples whose range is wider
    than one value, fraction unbounded)."""
    ps_o, lo, hi, unb = ora["per_sample"], ora["lo"], ora["hi"], ora["unbounded"]
    ps_g = g["ps"]
    N, L = ps_o.shape[:2]
    col = np.mean(np.abs(ps_o), axis=(0, 2), keepdims=True)        # per lobe / value
    tol = REL * np.maximum(np.abs(ps_o), col)
    bnd = ~unb[..., None].repeat(6, axis=-1)
    bad = bnd & ((ps_g < lo - tol) | (ps_g > hi + tol))
    assert not bad.any(), (np.argwhere(bad)[:3], ps_g[bad][:3], lo[bad][:3], hi[bad][:3])
    assert unb.mean() <= max_unbounded, unb.mean()
    u = ~bnd
    if u.sum() >= 2:
        dg, do = ps_g[u], ps_o[u]
        se = np.sqrt(dg.var(ddof=1) / len(dg) + do.var(ddof=1) / len(do))
        assert abs(dg.mean() - do.mean()) <= 4 * se + REL * np.abs(do).mean(), (dg.mean(), do.mean(), se)
    # per point: the mean of the samples' ranges (an unbounded sample leaves
    # only the lower bound)
    S = spp
    lo_p = lo[:, :, :S].mean(2)
    hi_p = np.where(unb[:, :, :S].any(2)[..., None], np.inf, hi[:, :, :S].mean(2))
    K = L - 1
    flat_g = np.concatenate([g["Ld"], g["Ls0"].reshape(N, -1), g["Ls1"].reshape(N, -1)], 1)
    flat_lo = np.concatenate([lo_p[:, 0, :3], lo_p[:, 1:, :3].reshape(N, -1), lo_p[:, 1:, 3:].reshape(N, -1)], 1)
    flat_hi = np.concatenate([hi_p[:, 0, :3], hi_p[:, 1:, :3].reshape(N, -1), hi_p[:, 1:, 3:].reshape(N, -1)], 1)
    assert flat_g.shape[1] == 3 + 6 * K
    flat_o = ora["flat"]
    sc = REL * np.maximum(np.abs(flat_o), np.mean(np.abs(flat_o), axis=0, keepdims=True))
    assert np.all(flat_g >= flat_lo - sc) and np.all(flat_g <= flat_hi + sc), \
        np.argwhere((flat_g < flat_lo - sc) | (flat_g > flat_hi + sc))[:3]
    wide = (hi - lo > 0).any(-1)
    return float(wide.mean()), float(unb.mean())


def test_refine_mirror_floor_cornell(fipt):
    m = cornell_box()
    T = m.T
    a = np.full((T, 3), 0.8, np.float32)
    r = np.ones(T, np.float32)
    mt = np.zeros(T, np.float32)
    r[m.floor] = 0.05
    mt[m.floor] = 1.0
    q = surface_queries(m, 512, seed=4)
    g, ora = run_both(fipt, m, q, a, r, mt, 16)
    print(check(g, ora, 16, 0.01))


def test_refine_without_mis_equals_stage_one_on_rough_scene(fipt):
    m = cornell_box()
    T = m.T
    q = surface_queries(m, 300, seed=5)
    a, r, mt = np.full((T, 3), 0.5, np.float32), np.ones(T, np.float32), np.zeros(T, np.float32)
    sc = fipt.Scene.from_mesh(m)
    sc.set_materials(cu(a), cu(r), cu(mt))
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    ref = fipt.bake(sc, qt, SIGMA, 32, 16, seed=2)
    got = fipt.bake_refine(sc, qt, SIGMA, 32, 16, mis=False, seed=2)
    for x, y in zip(got, ref):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.allclose(x, y, rtol=1e-5, atol=1e-6 * np.abs(y).mean())


def test_refine_room_random_materials(fipt):
    m = procedural_room(1)
    T = m.T
    rng = np.random.default_rng(8)
    a = rng.uniform(0, 1, (T, 3)).astype(np.float32)
    r = rng.uniform(0.02, 1.0, T).astype(np.float32)
    mt = rng.uniform(0, 1, T).astype(np.float32)
    q = surface_queries(m, 192, seed=6)
    g, ora = run_both(fipt, m, q, a, r, mt, 8)
    print(check(g, ora, 8, 0.05))


def test_refine_ragged_and_empty(fipt):
    m = cornell_box()
    T = m.T
    a, r, mt = np.full((T, 3), 0.5, np.float32), np.full(T, 0.3, np.float32), np.zeros(T, np.float32)
    for N in (1, 33):
        q = surface_queries(m, N, seed=N)
        g, ora = run_both(fipt, m, q, a, r, mt, 4, max_depth=3)
        check(g, ora, 4, 0.05)
    sc = fipt.Scene.from_mesh(m)
    sc.set_materials(cu(a), cu(r), cu(mt))
    out = fipt.bake_refine(sc, torch.zeros((0, 10), device="cuda"), SIGMA, 4)
    assert out[0].shape == (0, 3)


def test_refine_stats_counters(fipt):
    """The instrumented refinement gives the same shadings and counts its
    rays: at least one per sample, and on an all-rough scene without MIS
    exactly the stage-1 bake's rays (no path continues, no shadow ray)."""
    m = cornell_box()
    T = m.T
    q = surface_queries(m, 500, seed=12)
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    sc = fipt.Scene.from_mesh(m)
    sc.set_materials(cu(np.full((T, 3), 0.5, np.float32)), cu(np.ones(T, np.float32)),
                     cu(np.zeros(T, np.float32)))
    for mis in (False, True):
        st = torch.zeros(4, dtype=torch.int64, device="cuda")
        a = fipt.bake_refine(sc, qt, SIGMA, 16, 8, mis=mis, seed=3, stats=st)
        b = fipt.bake_refine(sc, qt, SIGMA, 16, 8, mis=mis, seed=3)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        n_rays, n_nodes, n_tris, max_sp = st.cpu().tolist()
        st0 = torch.zeros(4, dtype=torch.int64, device="cuda")
        fipt.bake(sc, qt, SIGMA, 16, 8, seed=3, stats=st0)
        bake_rays = st0.cpu().tolist()[0]
        if mis:
            assert n_rays > bake_rays
        else:
            assert n_rays == bake_rays
        assert n_nodes > n_rays and 0 < max_sp <= 32
    st = torch.zeros(4, dtype=torch.int64, device="cuda")
    c = fipt.bake_refine(sc, qt, SIGMA, 16, 8, seed=3, per_sample=True, stats=st)
    for x, y in zip(c, b):
        assert torch.equal(x, y)
    assert st[0].item() == n_rays


CHUNK = 1 << 24        # samples per chunk of a refinement call (documented in fipt.h)


def test_refine_chunks(fipt):
    """A call larger than one chunk of samples equals its points refined in
    separate calls (chunks are runs of whole points, the Philox counters
    carry global point indices); one point whose samples exceed a chunk is
    refused."""
    m = cornell_box()
    T = m.T
    a, r, mt = np.full((T, 3), 0.5, np.float32), np.ones(T, np.float32), np.zeros(T, np.float32)
    r[m.floor] = 0.05
    sc = fipt.Scene.from_mesh(m)
    sc.set_materials(cu(a), cu(r), cu(mt))
    spp_d, spp_s = 16384, 8192                      # 16384 + 3 * 8192 = 40,960 samples per point
    N = 600                                         # 24,576,000 samples: two chunks
    cut = CHUNK // (spp_d + 3 * spp_s)              # points in the first chunk
    assert cut < N
    q = surface_queries(m, N, seed=21)
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    whole = fipt.bake_refine(sc, qt, SIGMA, spp_d, spp_s, seed=5)
    parts = [fipt.bake_refine(sc, qt[lo:hi], SIGMA, spp_d, spp_s, seed=5, point_base=lo)
             for lo, hi in ((0, cut), (cut, N))]
    fipt.context().sync_status()
    for k in range(3):
        assert torch.equal(whole[k], torch.cat([parts[0][k], parts[1][k]]))
    with pytest.raises(fipt.FiptError):
        fipt.bake_refine(sc, qt[:4], SIGMA, CHUNK, 1)  # CHUNK + 3 samples for one point


def test_refine_deep_paths_match_oracle(fipt):
    """Glossy walls (sigma = 0.3 < sigma_c) keep paths going until they
    reach the light or leave through the open side; with max_depth = 40
    some paths pass 16 vertices (the call then checks every 16 depths
    whether any path is left, and must go on)."""
    m = cornell_box()
    T = m.T
    a, r, mt = np.full((T, 3), 0.8, np.float32), np.full(T, 0.3, np.float32), np.zeros(T, np.float32)
    q = surface_queries(m, 48, seed=22)
    g, ora = run_both(fipt, m, q, a, r, mt, 4, max_depth=40)
    print(check(g, ora, 4, 0.4))
    sc = fipt.Scene.from_mesh(m)
    sc.set_materials(cu(a), cu(r), cu(mt))
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    d16 = fipt.bake_refine(sc, qt, SIGMA, 4, 4, seed=3, request_id=1, max_depth=16)
    d40 = fipt.bake_refine(sc, qt, SIGMA, 4, 4, seed=3, request_id=1, max_depth=40)
    assert any(not torch.equal(x, y) for x, y in zip(d16, d40))
    for x, y in zip(d40, (g["Ld"], g["Ls0"], g["Ls1"])):
        assert np.array_equal(x.cpu().numpy(), y)
