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
