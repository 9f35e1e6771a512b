"""Environment light for rays that leave the scene (Sec. 8 window light):
GPU bake and refinement vs the oracle, and the uniform-sky closed form."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import ETA_BAKE, bake_flat, check_bake
from workloads import cornell_box, surface_queries

pytestmark = pytest.mark.gpu
SIGMA = [0.02, 0.25, 1.0]


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sky(seed=0, H=24, W=48):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 3.0, (H, W, 3)).astype(np.float32)


def test_uniform_sky_over_ground_is_exact(fipt):
    V = np.array([[-100, 0, -100], [100, 0, -100], [100, 0, 100], [-100, 0, 100]], np.float32)
    F = np.array([[0, 2, 1], [0, 3, 2]], np.int32)
    z = np.zeros((2, 3), np.float32)
    sc = fipt.Scene(cu(V), cu(F), cu(z), cu(z))
    L = np.array([1.5, 0.7, 0.2], np.float32)
    env = cu(np.broadcast_to(L, (8, 16, 3)))
    sc.set_environment(env)
    rng = np.random.default_rng(1)
    n = 1000
    x = np.c_[rng.uniform(-5, 5, n), np.zeros(n), rng.uniform(-5, 5, n)].astype(np.float32)
    nrm = np.tile([[0, 1, 0]], (n, 1)).astype(np.float32)
    q = fipt.pack_queries(cu(x), cu(nrm), cu(nrm), cu(np.zeros(n, np.int32)))
    Ld, _, _ = fipt.bake(sc, q, SIGMA, 32, 4)
    assert np.allclose(Ld.cpu().numpy(), L, rtol=2e-6, atol=0)


def test_open_cornell_box_with_sky_matches_oracle(fipt):
    m = cornell_box()                        # open front: rays leave through it
    q = surface_queries(m, 2048, seed=3)
    env = sky(2)
    sc = fipt.Scene.from_mesh(m)
    sc.set_environment(cu(env))
    Ld, Ls0, Ls1 = fipt.bake(sc, fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"])),
                             SIGMA, 32, 32, seed=6)
    fipt.context().sync_status()
    S = O.OracleScene.from_mesh(m)
    S.set_environment(env)
    ora = S.bake(q, SIGMA, 32, 32, seed=6, eta=ETA_BAKE)
    print(check_bake(bake_flat(Ld.cpu().numpy(), Ls0.cpu().numpy(), Ls1.cpu().numpy()), ora))
    assert np.mean(np.abs(ora["Ld"])) > 0.2        # the sky contributes


def test_refinement_sees_the_sky(fipt):
    from test_gpu_refine import check
    m = cornell_box()
    T = m.T
    a = np.full((T, 3), 0.7, np.float32)
    r = np.ones(T, np.float32)
    mt = np.zeros(T, np.float32)
    r[m.floor] = 0.05
    mt[m.floor] = 1.0
    q = surface_queries(m, 256, seed=9)
    env = sky(4)
    sc = fipt.Scene.from_mesh(m)
    sc.set_environment(cu(env))
    sc.set_materials(cu(a), cu(r), cu(mt))
    qt = fipt.pack_queries(cu(q["x"]), cu(q["n"]), cu(q["wo"]), cu(q["tri"]))
    Ld, Ls0, Ls1, ps = fipt.bake_refine(sc, qt, SIGMA, 8, 8, seed=2, per_sample=True)
    fipt.context().sync_status()
    S = O.OracleScene.from_mesh(m)
    S.set_environment(env)
    ora = S.refine(q, SIGMA, 8, 8, a, r, mt, seed=2, eta=1e-5, per_sample=True, bounds=True)
    g = {"Ld": Ld.cpu().numpy(), "Ls0": Ls0.cpu().numpy(), "Ls1": Ls1.cpu().numpy(),
         "ps": ps.cpu().numpy().astype(np.float64)}
    print(check(g, ora, 8, 0.05))
