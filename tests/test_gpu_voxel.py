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
    ora = S.refine(q, SIGMA, 8, 8, a, r, mt, seed=4, eta=1e-5, per_sample=True)
    g = {"Ld": Ld.cpu().numpy(), "Ls0": Ls0.cpu().numpy(), "Ls1": Ls1.cpu().numpy(),
         "ps": ps.cpu().numpy().astype(np.float64)}
    print(check(g, ora, 0.9, 0.3))
