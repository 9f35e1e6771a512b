"""Pins for the oracle's factorized render (Eq. 5, 8), tone-mapped loss
(Eq. 14), its analytic gradient, the per-triangle error (Sec. 4.4) and the
pinhole first hits used to generate queries (CPU only)."""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from workloads import cornell_box, surface_queries

GRID = np.array([0.02, 0.1, 0.25, 0.5, 0.75, 1.0])


def test_render_worked_example():
    rows = np.array(read_golden("render_worked_example.txt"), np.float64)
    grid = [0.0, 1.0]
    Ld = np.array([[1, 2, 3]] * 3, np.float64)
    Ls0 = np.array([[[1] * 3, [3] * 3]] * 3, np.float64)
    Ls1 = np.array([[[0.5] * 3, [1.5] * 3]] * 3, np.float64)
    a = np.array([[0.5, 0.5, 0.5], [1, 0.2, 0], [0.3, 0.6, 0.9]])
    s = np.array([0.5, 1.0, 0.0])
    m = np.array([0.5, 1.0, 0.0])
    Lr, _ = O.render_forward(Ld, Ls0, Ls1, grid, a, s, m)
    assert np.allclose(Lr, rows, rtol=0, atol=1e-12)


def test_lerp_reads_table_exactly_at_nodes_and_clamps():
    rng = np.random.default_rng(0)
    K = len(GRID)
    Ls0 = rng.random((K + 2, K, 3))
    Ls1 = rng.random((K + 2, K, 3))
    Ld = np.zeros((K + 2, 3))
    a = np.zeros((K + 2, 3))
    m = np.zeros(K + 2)
    s = np.concatenate([GRID, [0.0, 1.5]])        # nodes, then below / above the grid
    Lr, _ = O.render_forward(Ld, Ls0, Ls1, GRID, a, s, m)
    for k in range(K):
        assert np.allclose(Lr[k], 0.04 * Ls0[k, k] + Ls1[k, k], atol=1e-15)
    assert np.allclose(Lr[K], 0.04 * Ls0[K, 0] + Ls1[K, 0])
    assert np.allclose(Lr[K + 1], 0.04 * Ls0[K + 1, K - 1] + Ls1[K + 1, K - 1])
    i, t, cl = O.lerp_segment(s, GRID)
    assert i.tolist() == [0, 1, 2, 3, 4, 4, 0, 4]  # interior nodes take the right segment
    assert cl.tolist() == [False] * K + [True, True]


def test_tonemap_reference_points():
    # Gamma(e^y - 1) = sRGB(y); sRGB(1) = 1, sRGB(0) = 0, and the two pieces
    # of the sRGB curve meet at y = 0.0031308 to within 1e-7.
    assert O.tonemap(0.0) == 0.0
    assert abs(O.tonemap(np.e - 1.0) - 1.0) < 1e-15
    y = 0.0031308
    lin = 12.92 * y
    pw = 1.055 * y ** (1 / 2.4) - 0.055
    assert abs(lin - pw) < 1e-7
    assert abs(O.tonemap(np.expm1(y)) - lin) < 1e-15
    assert O.tonemap(-3.0) == 0.0
    xs = np.array([1e-5, 0.01, 0.3, 2.0, 40.0])
    h = 1e-7
    fd = (O.tonemap(xs + h) - O.tonemap(xs - h)) / (2 * h)
    assert np.allclose(O.tonemap_grad(xs), fd, rtol=1e-6)


def _per_point_loss(Ld, Ls0, Ls1, a, s, m, Lgt):
    Lr, _ = O.render_forward(Ld, Ls0, Ls1, GRID, a, s, m)
    return np.sum((O.tonemap(Lr) - O.tonemap(Lgt)) ** 2, axis=1)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    N, K = 4000, len(GRID)
    Ld = rng.uniform(0, 3, (N, 3))
    Ls0 = rng.uniform(0, 3, (N, K, 3))
    Ls1 = rng.uniform(0, 0.5, (N, K, 3))
    a = rng.uniform(0, 1, (N, 3))
    s = rng.uniform(0.0, 1.0, N)          # includes sigma < 0.02 (clamped)
    m = rng.uniform(0, 1, N)
    Lgt = rng.uniform(0, 3, (N, 3))
    h = 1e-6
    ga, gs, gm = O.render_grad(Ld, Ls0, Ls1, GRID, a, s, m, Lgt)
    Lr, _ = O.render_forward(Ld, Ls0, Ls1, GRID, a, s, m)
    y = np.log1p(np.maximum(Lr, 0))
    near_knee = np.any(np.abs(y - 0.0031308) < 1e-3, axis=1)
    near_node = np.min(np.abs(s[:, None] - GRID[None, :]), axis=1) < 4 * h
    ok = ~near_knee & ~near_node
    f = lambda a_, s_, m_: _per_point_loss(Ld, Ls0, Ls1, a_, s_, m_, Lgt)
    for c in range(3):
        e = np.zeros_like(a)
        e[:, c] = h
        fd = (f(a + e, s, m) - f(a - e, s, m)) / (2 * h)
        assert np.allclose(ga[ok, c], fd[ok], rtol=1e-6, atol=1e-8)
    fd = (f(a, s + h, m) - f(a, s - h, m)) / (2 * h)
    assert np.allclose(gs[ok], fd[ok], rtol=1e-6, atol=1e-8)
    assert np.all(gs[s < GRID[0] - 4 * h] == 0.0)
    fd = (f(a, s, m + h) - f(a, s, m - h)) / (2 * h)
    assert np.allclose(gm[ok], fd[ok], rtol=1e-6, atol=1e-8)


def test_loss_mask_and_grad_scale():
    rng = np.random.default_rng(2)
    N, K = 50, len(GRID)
    args = (rng.random((N, 3)), rng.random((N, K, 3)), rng.random((N, K, 3)), GRID,
            rng.random((N, 3)), rng.uniform(0.02, 1, N), rng.random(N))
    Lgt = rng.random((N, 3))
    mask = rng.random(N) < 0.5
    _, full = O.render_forward(*args, Lgt=Lgt)
    _, part = O.render_forward(*args, Lgt=Lgt, mask=mask)
    _, rest = O.render_forward(*args, Lgt=Lgt, mask=~mask)
    assert abs(full - part - rest) < 1e-12
    g1 = O.render_grad(*args, Lgt, mask=mask)
    g2 = O.render_grad(*args, Lgt, mask=mask, grad_scale=-2.5)
    for x, y in zip(g1, g2):
        assert np.allclose(-2.5 * x, y)
        assert np.all(x[~mask] == 0)


def test_tri_error_worked_example():
    rows = np.array(read_golden("tri_error_worked_example.txt"), np.float64)
    tri = np.array([2, 0, 2, -1, 0])
    Lr = np.array([[1, 1, 1], [1, 2, 3], [0, 0, 0], [9, 9, 9], [2, 2, 2]], np.float64)
    Lgt = np.array([[1, 1, 1], [0, 0, 0], [0.5, 0, 0], [0, 0, 0], [1, 1, 1]], np.float64)
    err, cnt = O.tri_error(tri, Lr, Lgt, 3)
    assert np.allclose(err, rows[:, 1], atol=0)
    assert cnt.tolist() == rows[:, 2].astype(int).tolist()


def test_tri_error_conserves_totals():
    rng = np.random.default_rng(3)
    P, T = 10000, 300
    tri = rng.integers(-1, T, P)
    Lr, Lgt = rng.random((P, 3)), rng.random((P, 3))
    err, cnt = O.tri_error(tri, Lr, Lgt, T)
    v = tri >= 0
    assert cnt.sum() == v.sum()
    assert abs(err.sum() - np.sum((Lr[v] - Lgt[v]) ** 2)) < 1e-9


def test_camera_first_hit_reprojects_to_its_pixel():
    m = cornell_box(closed=True)
    S = O.OracleScene.from_mesh(m)
    cam = np.array([[0.5, 0.5, 0.3, 0.1, -0.05, 1.0, 0, 1, 0, np.deg2rad(60.0)]], np.float32)
    W, H = 32, 24
    pix = np.arange(W * H)
    q = S.camera_queries(cam, W, H, pix)
    assert np.all(q["tri"] >= 0)
    eye = cam[0, :3].astype(np.float64)
    fwd = cam[0, 3:6].astype(np.float64)
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, [0, 1.0, 0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    th = np.tan(0.5 * float(cam[0, 9]))
    v = q["x"] - eye
    z = v @ fwd
    px = ((v @ right) / z / (th * W / H) + 1) * W / 2 - 0.5
    py = (1 - (v @ up) / z / th) * H / 2 - 0.5
    assert np.allclose(px, pix % W, atol=1e-9)
    assert np.allclose(py, pix // W, atol=1e-9)
    assert np.allclose(q["wo"], -v / np.linalg.norm(v, axis=1, keepdims=True))
    # normals face the camera and are unit length
    assert np.all(np.sum(q["n"] * q["wo"], 1) > 0)
    assert np.allclose(np.linalg.norm(q["n"], axis=1), 1.0)
    # every hit point lies on its triangle's plane
    V = m.V.astype(np.float64)
    v0 = V[m.F[q["tri"], 0]]
    assert np.allclose(np.sum((q["x"] - v0) * q["n"], 1), 0, atol=1e-12)


def test_specular_terms_vanish_at_grazing_view():
    # reading of Sec. 3: 1/(n.wo) is not evaluated for n.wo <= 1e-2; the point
    # gets zero specular shading and keeps its diffuse shading.
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    mu = 0.005
    q = {"x": np.array([[0.5, 0.0, 0.6]], np.float32), "n": np.array([[0, 1, 0]], np.float32),
         "wo": np.array([[np.sqrt(1 - mu * mu), mu, 0]], np.float32),
         "tri": np.array([-1], np.int32)}
    r = S.bake(q, GRID, 64, 64)
    assert np.all(r["Ls0"] == 0) and np.all(r["Ls1"] == 0)
    assert np.all(r["Ld"] > 0)
