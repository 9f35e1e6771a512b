"""Pins for the oracle's emitter extraction (Sec. 4.4, Eq. 12), CPU only.

* Sampling: the points are uniform on the triangle, checked through their
  barycentric moments (E b_i = 1/3, E b_i^2 = 1/6, E b_i b_j = 1/12 for the
  uniform distribution on a simplex) recovered independently from the
  points by solving for the barycentrics.
* Classification and the median: a hand-worked example.
* The closed form: the returned L_e minimises the L1 loss of Eq. 12 (with
  L_r = 0 at an emitter) over every candidate value, by brute force.
"""
import numpy as np

import oracle as O
from conftest import read_golden
from workloads import cornell_box, emitter_pixels


def one_triangle(v0, v1, v2):
    V = np.array([v0, v1, v2], np.float32)
    return O.OracleScene(V, np.array([[0, 1, 2]], np.int32))


def barycentrics(V, x):
    e1, e2 = V[1] - V[0], V[2] - V[0]
    A = np.stack([e1, e2], 1)                     # 3 x 2
    b12, *_ = np.linalg.lstsq(A, (x - V[0]).T, rcond=None)
    b = np.vstack([1 - b12.sum(0), b12]).T
    resid = np.linalg.norm(V[0] + (A @ b12).T - x, axis=1)
    return b, resid


def test_points_are_uniform_on_the_triangle():
    V = np.array([[0.2, -1.0, 0.5], [3.0, 0.5, -0.7], [-0.4, 2.0, 1.1]])
    S = one_triangle(*V)
    n = 200000
    x = S.emitter_points(n, seed=9, request_id=3)
    b, resid = barycentrics(V.astype(np.float32).astype(np.float64), x)
    assert resid.max() < 1e-12 and b.min() > -1e-12
    assert np.allclose(b.sum(1), 1.0)
    tol = 5.0 / np.sqrt(n)
    assert np.all(np.abs(b.mean(0) - 1 / 3) < tol * 0.25), b.mean(0)
    assert np.all(np.abs((b ** 2).mean(0) - 1 / 6) < tol * 0.25), (b ** 2).mean(0)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert abs((b[:, i] * b[:, j]).mean() - 1 / 12) < tol * 0.15
    # a quarter of the area (the sub-triangle at v0 cut at half the edges)
    # holds a quarter of the points
    frac = np.mean(b[:, 1] + b[:, 2] < 0.5)
    assert abs(frac - 0.25) < 5 * np.sqrt(0.25 * 0.75 / n)


def test_points_depend_on_seed_and_request_only_through_the_counter():
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    a = S.emitter_points(7, seed=1, request_id=0)
    b = S.emitter_points(7, seed=1, request_id=0)
    c = S.emitter_points(7, seed=2, request_id=0)
    d = S.emitter_points(7, seed=1, request_id=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c) and not np.array_equal(a, d)
    assert a.shape == (m.T * 7, 3)
    # point j of triangle t lies on triangle t
    V = m.V.astype(np.float64)
    for t in (0, 5, m.T - 1):
        bt, res = barycentrics(V[m.F[t]], a[7 * t:7 * t + 7])
        assert res.max() < 1e-12 and bt.min() > -1e-12


def golden():
    rows = read_golden("emitter_extraction_worked_example.txt")
    alpha = np.array([[float(v) for v in r[2:]] for r in rows if r[0] == "alpha"], np.float32)
    pix = [r[1:] for r in rows if r[0] == "pixel"]
    tri = np.array([int(r[0]) for r in pix], np.int32)
    rgb = np.array([[float(v) for v in r[1:]] for r in pix], np.float32)
    want = np.array([[float(v) for v in r[1:]] for r in rows if r[0] == "want"])
    return alpha, tri, rgb, want


def test_worked_example():
    alpha, tri, rgb, want = golden()
    flag, mean = O.emitter_classify(alpha.reshape(-1), 4, 0.01)
    assert flag.tolist() == want[:, 1].astype(int).tolist()
    Le, cnt = O.emitter_radiance(tri, rgb, flag)
    assert cnt.tolist() == want[:, 2].astype(int).tolist()
    assert np.array_equal(Le, want[:, 3:6].astype(np.float32))


def test_median_minimises_the_l1_loss_of_eq12():
    rng = np.random.default_rng(4)
    T = 40
    flag = (rng.uniform(size=T) < 0.7).astype(np.uint8)
    P = 3000
    tri = rng.integers(-3, T, P).astype(np.int32)
    rgb = (rng.lognormal(0.0, 1.0, (P, 3)) * rng.choice([1, -1], (P, 3), p=[0.9, 0.1])).astype(np.float32)
    rgb[rng.uniform(size=P) < 0.05] *= 50.0          # outliers (highlights)
    Le, cnt = O.emitter_radiance(tri, rgb, flag)
    for t in range(T):
        sel = rgb[tri == t].astype(np.float64)
        if not flag[t]:
            assert cnt[t] == 0 and np.all(Le[t] == 0)
            continue
        assert cnt[t] == len(sel)
        if len(sel) == 0:
            assert np.all(Le[t] == 0)
            continue
        for c in range(3):
            v = sel[:, c]
            cand = np.unique(np.concatenate([v, (v[:, None] + v[None, :]).ravel() / 2]))
            loss = np.abs(cand[:, None] - v[None, :]).sum(1)
            got = np.abs(float(Le[t, c]) - v).sum()
            assert got <= loss.min() * (1 + 1e-12), (t, c)
            # and it is the lower of the two middle values
            k = int(np.sum(v < Le[t, c])), int(np.sum(v <= Le[t, c]))
            assert k[0] <= (len(v) - 1) // 2 < k[1]


def test_median_is_robust_on_a_synthetic_capture():
    m = cornell_box()
    tri, rgb = emitter_pixels(m, 200000, seed=5)
    Le, cnt = O.emitter_radiance(tri, rgb, m.emitter.astype(np.uint8))
    e = np.nonzero(m.emitter)[0]
    assert np.all(cnt[e] > 1000)
    # pixel noise is a multiplicative lognormal with median 1 plus 5% bright
    # outliers: the median recovers L_e to a few percent
    assert np.allclose(Le[e], m.Le[e], rtol=0.03)
    assert not np.any(Le[~m.emitter])


def test_classify_threshold_is_strict_and_fp64():
    n = 100
    a = np.zeros((3, n), np.float32)
    a[0, 0] = np.float32(1.0)          # mean 0.01 in FP64 of f32(1)/100 -> exactly 0.01
    a[1, 0] = np.float32(1.01)         # mean 0.0101
    a[2, :] = np.float32(0.01)         # mean = f32(0.01) = 0.0099999998 < 0.01 (double)
    flag, mean = O.emitter_classify(a.reshape(-1), n, 0.01)
    # threshold 0.01 as f32 is 0.009999999776...; 0.01 > it, f32(0.01) mean equals it
    assert flag.tolist() == [1, 1, 0]
    assert mean[2] == float(np.float32(0.01))
