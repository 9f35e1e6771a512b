"""Pins for the oracle's voxel radiance cache (Sec. 4.2), CPU only: a
hand-worked pooling example, and a furnace whose cache is pooled from
uniform-radiance pixels covering every surface (L_d = L exactly)."""
import numpy as np

import oracle as O
from conftest import read_golden
from workloads import cornell_box, surface_queries


def box_scene():
    pts = [(0, 0, 0), (2, 2, 2)]
    V = np.array([p for p in pts for _ in range(3)], np.float32)
    F = np.arange(6, dtype=np.int32).reshape(2, 3)
    return O.OracleScene(V, F)


def test_pooling_worked_example():
    S = box_scene()
    x = np.array([[0.5, 0.5, 0.5], [0.25, 0.75, 0.1], [1.5, 0.5, 0.5], [2, 2, 2]], np.float32)
    L = np.array([[1, 2, 3], [3, 2, 1], [4, 0, 0], [0, 0, 6]], np.float32)
    g = S.voxel_pool(x, L, 2).reshape(-1, 4)
    want = np.zeros((8, 4))
    for row in read_golden("voxel_pool_worked_example.txt"):
        want[int(row[0])] = [float(v) for v in row[1:]]
    assert np.array_equal(g, want)


def test_furnace_with_pooled_cache():
    L = 0.6
    m = cornell_box(closed=True, furnace_radiance=L)
    S = O.OracleScene.from_mesh(m)
    px = surface_queries(m, 200000, seed=1, all_triangles=True)["x"]
    # R = 7: no face of the box's geometry lies on a cell face (with R = 8
    # the tall box's z = 0.5 face would, and its hits would fall on either side)
    grid = S.voxel_pool(px, np.full((len(px), 3), L, np.float32), 7)
    S.set_voxel_cache(grid)
    q = surface_queries(m, 64, seed=2)
    r = S.bake(q, [0.5], 64, 4)
    assert np.max(np.abs(r["Ld"] - float(np.float32(L)))) < 1e-12
    # an empty grid brings no cache light at all
    S.set_voxel_cache(np.zeros_like(grid))
    assert np.all(S.bake(q, [0.5], 16, 4)["Ld"] == 0)
