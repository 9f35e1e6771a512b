"""Voxel radiance cache (Sec. 4.2) on the GPU vs the oracle: pooling (voxel
of every pixel decided in correctly rounded FP64 on both sides, means summed
in pixel order, so the float32 grid is the oracle's rounded value exactly),
then the bake and the refinement reading the cache at hit points."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import ETA_BAKE, bake_flat, check_bake
from workloads import cornell_box, procedural_room, surface_queries

pytestmark = pytest.mark.gpu
SIGMA = [0.02, 0.25, 1.0]


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pixels(m, P, seed):
    """First-hit points on every triangle with a per-triangle radiance plus
    per-pixel noise (what a captured image pooled onto the surface looks like)."""
    q = surface_queries(m, P, seed=seed, all_triangles=True)
    rng = np.random.default_rng(seed + 100)
    base = rng.uniform(0.0, 2.0, (m.T, 3))
    L = base[q["tri"]] * rng.uniform(0.8, 1.2, (P, 3))
    return q, L.astype(np.float32)


@pytest.mark.parametrize("R", [1, 7, 64, 256])
def test_pool_matches_oracle_exactly(fipt, R):
    m = procedural_room(1)
    q, L = pixels(m, 300000, 1)
    # a few pixels outside the scene box clamp to the border voxels
    x = q["x"].copy()
    x[:7] += np.float32(50.0)
    x[7:14] -= np.float32(50.0)
    sc = fipt.Scene.from_mesh(m)
    g = sc.voxel_cache(cu(x), cu(L), R).cpu().numpy()
    o = O.OracleScene.from_mesh(m).voxel_pool(x, L, R)
    assert np.array_equal(g[..., 3], o[..., 3])                     # counts
    assert np.array_equal(g, o.astype(np.float32))                  # means
    assert o[..., 3].sum() == len(x)


@pytest.mark.parametrize("R", [64, 128])
def test_pool_cell_faces_match_oracle(fipt, R):
    """Pixels exactly on a cell face and 1-2 float32 ulps either side of it,
    on every axis: the cell is decided in correctly rounded FP64 on both
    sides, and those pixels are the ones a float32 estimate cannot place."""
    m = cornell_box()
    V = np.asarray(m.V, np.float32)
    lo, hi = V.min(0).astype(np.float64), V.max(0).astype(np.float64)
    rng = np.random.default_rng(R)
    n = 6000
    k = rng.integers(0, R + 1, (n, 3))
    x = (lo + k * (hi - lo) / R).astype(np.float32)
    for step in (-2, -1, 1, 2):
        sel = rng.random((n, 3)) < 0.2
        for _ in range(abs(step)):
            x = np.where(sel, np.nextafter(x, np.float32(np.inf if step > 0 else -np.inf)), x)
    x = np.concatenate([x, rng.uniform(lo, hi, (4000, 3)).astype(np.float32)])
    L = rng.uniform(0.0, 2.0, (len(x), 3)).astype(np.float32)
    g = fipt.Scene.from_mesh(m).voxel_cache(cu(x), cu(L), R).cpu().numpy()
    o = O.OracleScene.from_mesh(m).voxel_pool(x, L, R)
    assert np.array_equal(g[..., 3], o[..., 3])
    assert np.array_equal(g, o.astype(np.float32))


def test_pool_degenerate_extent_matches_oracle(fipt):
    """A scene box whose z extent is the subnormal 1e-39: R / extent is
    larger than any float32, so every pixel's z cell comes from the FP64
    arithmetic; the x and y axes keep the float32 route."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1e-39], [1, 1, 1e-39]], np.float32)
    F = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    z = np.array([0.0, 1e-45, 1e-40, 2.5e-40, 3e-40, 5e-40, 7.5e-40, 1e-39, 2e-39, -1e-45], np.float32)
    rng = np.random.default_rng(4)
    n = 4000
    x = np.stack([rng.uniform(0, 1, n), rng.uniform(0, 1, n), rng.choice(z, n)], 1).astype(np.float32)
    L = rng.uniform(0, 2, (n, 3)).astype(np.float32)
    sc = fipt.Scene(cu(V), cu(F), cu(np.zeros((2, 3), np.float32)), cu(np.zeros((2, 3), np.float32)))
    for R in (4, 16):
        g = sc.voxel_cache(cu(x), cu(L), R).cpu().numpy()
        o = O.OracleScene(V, F).voxel_pool(x, L, R)
        assert np.array_equal(g, o.astype(np.float32))
        assert (o[..., 3].sum(axis=(1, 2)) > 0).sum() >= 3          # several z layers are occupied


def test_pool_mixed_magnitudes_match_oracle(fipt):
    """Voxels whose pixels mix zeros, both signs, subnormals, infinities,
    NaNs and magnitudes far apart (sums that leave the range in which the
    in-order FP64 sum is exact), interleaved with ordinary pixels: the mean
    is the oracle's in-order FP64 sum over the count, rounded to float32."""
    m = cornell_box()
    V = np.asarray(m.V, np.float32)
    lo, hi = V.min(0), V.max(0)
    R = 16
    f = np.float32
    special = [
        [1.0, 1.5, 2.0 ** -29],                    # magnitudes reach 2^53 units
        [1e-12, 1e3, 7.0],                         # exponents 50 apart
        [0.0, -0.0, 0.0],                          # zeros only: +0
        [3.0, -3.0, 1e-3, -1e-3],                  # cancellations
        [1e-40, 1.0, 2e-45],                       # subnormals
        [np.inf, 1.0], [np.inf, -np.inf], [np.nan, 2.0],
        [2.0 ** -100, 2.0 ** -110, 3 * 2.0 ** -120],  # tiny normals, exact
        [-(2.0 ** 20), 2.0 ** -9, 2.0 ** 20],      # exact: 2^20 - 2^20 + 2^-9
        list(np.random.default_rng(1).uniform(0.5, 2.0, 5000)),   # one long run
    ]
    rng = np.random.default_rng(2)
    xs, Ls = [], []
    for i, vals in enumerate(special):
        cell = np.array([i % R, (i // R) % R, 3], np.float64) + 0.5
        p = (lo + cell * (hi - lo) / R).astype(np.float32)
        vv = np.array(vals, np.float32)
        Lv = np.stack([vv, vv[::-1], rng.permutation(vv)], 1)   # each channel its own order
        xs.append(np.repeat(p[None], len(vv), 0))
        Ls.append(Lv)
    xs.append(rng.uniform(lo, hi, (3000, 3)).astype(f))
    Ls.append(rng.uniform(0.0, 2.0, (3000, 3)).astype(f))
    x = np.concatenate(xs)
    L = np.concatenate(Ls).astype(f)
    perm = rng.permutation(len(x))                   # interleave the voxels' pixels
    x, L = x[perm], L[perm]
    g = fipt.Scene.from_mesh(m).voxel_cache(cu(x), cu(L), R).cpu().numpy()
    o = O.OracleScene.from_mesh(m).voxel_pool(x, L, R)
    assert np.array_equal(g[..., 3], o[..., 3])
    with np.errstate(invalid="ignore", over="ignore"):
        o32 = o.astype(np.float32)
    assert np.array_equal(g.view(np.uint32)[~np.isnan(g)], o32.view(np.uint32)[~np.isnan(o32)])
    assert np.array_equal(np.isnan(g), np.isnan(o32))


def test_pool_from_query_records_and_empty(fipt):
    m = cornell_box()
    q, L = pixels(m, 5000, 2)
    sc = fipt.Scene.from_mesh(m)
    rec = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    a = sc.voxel_cache(rec, cu(L), 16).cpu().numpy()
    b = sc.voxel_cache(cu(q["x"]), cu(L), 16).cpu().numpy()
    assert np.array_equal(a, b)
    e = sc.voxel_cache(torch.zeros((0, 3), device="cuda"), torch.zeros((0, 3), device="cuda"), 4)
    assert e.shape == (4, 4, 4, 4) and not e.any()
    S = O.OracleScene.from_mesh(m)
    for P in (1, 33, 1025):                       # one pixel; ragged tiles of the run-head scan
        g = sc.voxel_cache(cu(q["x"][:P]), cu(L[:P]), 16).cpu().numpy()
        assert np.array_equal(g, S.voxel_pool(q["x"][:P], L[:P], 16).astype(np.float32))


def bake_both(fipt, m, grid_R, spp_d, spp_s, nq, seed):
    q, L = pixels(m, 400000, seed)
    sc = fipt.Scene.from_mesh(m)
    sc.set_voxel_cache(sc.voxel_cache(cu(q["x"]), cu(L), grid_R))
    qq = surface_queries(m, nq, seed=seed + 1)
    Ld, Ls0, Ls1 = fipt.bake(sc, fipt.pack_queries(cu(qq["x"]), cu(qq["n"]), cu(qq["wo"]), cu(qq["tri"])),
                             SIGMA, spp_d, spp_s, seed=seed)
    fipt.context().sync_status()
    S = O.OracleScene.from_mesh(m)
    S.set_voxel_cache(S.voxel_pool(q["x"], L, grid_R))
    ora = S.bake(qq, SIGMA, spp_d, spp_s, seed=seed, eta=ETA_BAKE)
    return bake_flat(Ld.cpu().numpy(), Ls0.cpu().numpy(), Ls1.cpu().numpy()), ora


@pytest.mark.parametrize("R", [24, 256])
def test_bake_with_voxel_cache_matches_oracle(fipt, R):
    g, ora = bake_both(fipt, procedural_room(1), R, 32, 16, 1500, 5)
    print(check_bake(g, ora))
    assert np.mean(np.abs(ora["Ld"])) > 0.05


def test_bake_cornell_voxel_cache_matches_oracle(fipt):
    g, ora = bake_both(fipt, cornell_box(), 32, 64, 32, 1024, 6)
    print(check_bake(g, ora))


def test_refine_reads_voxel_cache(fipt):
    from test_gpu_refine import check
    m = cornell_box()
    T = m.T
    a = np.full((T, 3), 0.6, np.float32)
    r = np.ones(T, np.float32)
    mt = np.zeros(T, np.float32)
    r[m.floor] = 0.05
    mt[m.floor] = 1.0
    qp, L = pixels(m, 200000, 7)
    sc = fipt.Scene.from_mesh(m)
    sc.set_voxel_cache(sc.voxel_cache(cu(qp["x"]), cu(L), 32))
    sc.set_materials(cu(a), cu(r), cu(mt))
    q = surface_queries(m, 256, seed=8)
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    Ld, Ls0, Ls1, ps = fipt.bake_refine(sc, qt, SIGMA, 8, 8, seed=4, per_sample=True)
    fipt.context().sync_status()
    S = O.OracleScene.from_mesh(m)
    S.set_voxel_cache(S.voxel_pool(qp["x"], L, 32))
    ora = S.refine(q, SIGMA, 8, 8, a, r, mt, seed=4, eta=1e-5, per_sample=True, bounds=True)
    g = {"Ld": Ld.cpu().numpy(), "Ls0": Ls0.cpu().numpy(), "Ls1": Ls1.cpu().numpy(),
         "ps": ps.cpu().numpy().astype(np.float64)}
    print(check(g, ora, 8, 0.05))
