"""Pins for rays that leave the scene and see the environment (window light,
Sec. 8), CPU only.  A point on a large ground plane looking up sees only
sky, so:
  * a uniform sky L gives L_d = L exactly and L_s0 + L_s1 = L (A + B), the
    GGX white-furnace quadrature of the BRDF;
  * a sky that is linear in colatitude between the first and last texel
    rows (bilinear lookup reproduces it exactly) gives
    L_d = 2 int_0^{pi/2} env(theta) cos(theta) sin(theta) d theta.
"""
import numpy as np
from scipy import integrate

import oracle as O
from test_oracle_bake import white_furnace_AB

SIGMA = [0.25, 0.5, 1.0]


def ground():
    V = np.array([[-100, 0, -100], [100, 0, -100], [100, 0, 100], [-100, 0, 100]], np.float32)
    F = np.array([[0, 2, 1], [0, 3, 2]], np.int32)           # facing +y
    return O.OracleScene(V, F, np.zeros((2, 3)), np.zeros((2, 3)))


def up_query(mu_o=1.0):
    wo = [np.sqrt(1 - mu_o ** 2), mu_o, 0.0]
    return {"x": np.array([[0.3, 0.0, -0.2]], np.float32), "n": np.array([[0, 1, 0]], np.float32),
            "wo": np.array([wo], np.float32), "tri": np.array([0], np.int32)}


def test_uniform_sky():
    S = ground()
    L = np.array([1.5, 0.7, 0.2], np.float32)
    S.set_environment(np.broadcast_to(L, (16, 32, 3)))
    for mu in (1.0, 0.4):
        outs = [S.bake(up_query(mu), SIGMA, 64, 2048, seed=2, request_id=b)["flat"][0] for b in range(8)]
        a = np.array(outs)
        assert np.all(a[:, :3] == L.astype(np.float64))       # every ray sees the sky
        mean, se = a.mean(0), a.std(0, ddof=1) / np.sqrt(len(a))
        K = len(SIGMA)
        for k, s in enumerate(SIGMA):
            A, B = white_furnace_AB(mu, s * s, 512, 256)
            tot = mean[3 + 3 * k: 6 + 3 * k] + mean[3 + 3 * K + 3 * k: 6 + 3 * K + 3 * k]
            err = se[3 + 3 * k: 6 + 3 * k] + se[3 + 3 * K + 3 * k: 6 + 3 * K + 3 * k]
            assert np.all(np.abs(tot - L * (A + B)) <= 4 * err + 1e-6)


def test_sky_linear_in_colatitude():
    S = ground()
    H, W = 64, 8
    a, b = 2.0, -1.5
    v = (np.arange(H) + 0.5) / H
    rows = a + b * v
    env = np.repeat(np.repeat(rows[:, None, None], W, 1), 3, 2).astype(np.float32)
    S.set_environment(env)

    def sky(theta):
        vv = np.clip(theta / np.pi, 0.5 / H, 1 - 0.5 / H)
        return a + b * vv
    ref = 2 * integrate.quad(lambda t: sky(t) * np.cos(t) * np.sin(t), 0, np.pi / 2,
                             points=[np.pi * 0.5 / H], epsabs=1e-13)[0]
    outs = [S.bake(up_query(), [0.5], 4096, 1, seed=4, request_id=i)["flat"][0, :3] for i in range(16)]
    o = np.array(outs)
    mean, se = o.mean(0), o.std(0, ddof=1) / np.sqrt(len(o))
    assert np.all(np.abs(mean - ref) <= 4 * se + 1e-9), (mean, ref, se)
    # without the sky every ray misses into darkness
    S.set_environment(None)
    assert np.all(S.bake(up_query(), [0.5], 64, 4)["flat"] == 0)


GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                    "env_lookup_worked_example.txt")


def _golden_rows():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            kind, a, b, c, e0, e1, e2 = line.split()
            if kind == "dir":
                d = np.array([float(a), float(b), float(c)])
            else:              # (u, v) -> the direction whose longitude / colatitude they are
                phi, th = 2 * np.pi * (float(a) - 0.5), np.pi * float(b)
                d = np.array([np.sin(th) * np.sin(phi), np.cos(th), -np.sin(th) * np.cos(phi)])
            rows.append((d, np.array([float(e0), float(e1), float(e2)])))
    return rows


def test_lookup_worked_example():
    """Hand-computed bilinear lookups of an 8 x 4 map (tests/golden): axis
    directions, the seam, the pole, the bottom clamp and a single-texel
    impulse.  A swapped or negated atan2 argument moves the +x / -x rows; a
    half-texel offset moves every row; a missing wrap breaks the seam rows."""
    S = ground()
    W, H = 8, 4
    env = np.zeros((H, W, 3), np.float32)
    for j in range(H):
        for i in range(W):
            env[j, i] = (i + 10 * j, 1.0 if (i, j) == (5, 1) else 0.0, j)
    S.set_environment(env)
    rows = _golden_rows()
    got = S.env_lookup(np.array([d for d, _ in rows]))
    for (d, e), g in zip(rows, got):
        assert np.allclose(g, e, rtol=0, atol=1e-9), (d, g, e)
    S.set_environment(None)
    assert np.all(S.env_lookup(np.array([[0.0, 0.0, -1.0]])) == 0)


def _far_speck():
    """A scene whose only triangle lies far below: every ray from the origin
    region upward or sideways leaves the scene."""
    V = np.array([[-1e-3, -1e4, 0], [1e-3, -1e4, 0], [0, -1e4, 1e-3]], np.float32)
    return O.OracleScene(V, np.array([[0, 1, 2]], np.int32), np.zeros((1, 3)), np.zeros((1, 3)))


def test_sky_varying_in_longitude_only():
    """Skies that depend on longitude alone (texel centres of a 4096-wide
    map, so bilinear reproduces them to ~1e-7), every ray leaving the scene.
    With phi = 2 pi (u - 1/2), the reading makes sin phi = d.x / rho and
    cos phi = -d.z / rho (rho = |(d.x, d.z)|), so env = 1 + 0.5 sin phi seen
    from a point facing +x and env = 1 + 0.5 cos phi seen from a point
    facing -z both give L_d = 1 + 0.5 I / pi, I = int_hemisphere
    (n.d)^2 / rho d omega (one I for both, by x <-> z symmetry), computed
    here by 2-D quadrature.  Swapping the two atan2 arguments makes the
    varying term odd over the hemisphere (L_d = 1); negating one argument or
    dropping the 1/2 shift gives 1 - 0.5 I / pi."""
    from scipy import integrate
    S = _far_speck()
    W = 4096
    phi = 2 * np.pi * ((np.arange(W) + 0.5) / W - 0.5)
    I = integrate.dblquad(lambda a, b: np.cos(a) ** 2 * np.sin(a) /
                          np.sqrt(np.cos(a) ** 2 + (np.sin(a) * np.sin(b)) ** 2),
                          0, 2 * np.pi, 0, np.pi / 2, epsabs=1e-11, epsrel=1e-11)[0]
    ref = 1.0 + 0.5 * I / np.pi
    for n, wave in (([1, 0, 0], np.sin), ([0, 0, -1], np.cos)):
        row = 1.0 + 0.5 * wave(phi)
        S.set_environment(np.repeat(np.repeat(row[None, :, None], 2, 0), 3, 2).astype(np.float32))
        wo = n
        npts = 64
        q = {"x": np.zeros((npts, 3), np.float32), "n": np.tile(np.array(n, np.float32), (npts, 1)),
             "wo": np.tile(np.array(wo, np.float32), (npts, 1)), "tri": np.full(npts, -1, np.int32)}
        o = S.bake(q, [0.5], 4096, 1, seed=6)["flat"][:, 0]
        mean, se = o.mean(), o.std(ddof=1) / np.sqrt(len(o))
        assert abs(mean - ref) <= 4 * se + 1e-6, (n, mean, ref, se)
