"""Pins for the oracle's bake (Eq. 6, 7 estimated as in Sec. 6, stage 1,
through the one-segment cache query of Eq. 9), CPU only.

Each pin compares the Monte Carlo estimator with something it does not
compute itself:
  * furnace: a closed enclosure of uniform radiance L gives L_d = L exactly;
  * white furnace: L_s0 / L_s1 in that enclosure equal deterministic
    quadratures of the GGX BRDF of Eq. 1 (explicit D, G, F; no sampling);
  * GGX normalisation: the projected D integrates to one;
  * Lambert's closed-form point-to-polygon form factor under the emitter;
  * one-sided emission: a point that only sees the emitter's back is dark;
  * brute-force hemisphere quadrature of L_d and L_s on the occluded
    Cornell box (rays cast by brute force, radiance looked up here).
Statistical pins use batch means: the estimate is the mean of B independent
request streams and must agree within 4 standard errors of that mean plus
the quadrature's own error (estimated from two resolutions).
"""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss
from scipy import integrate

import oracle as O
from workloads import cornell_box, surface_queries

SIGMA = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]


# ----------------------------------------------------------------- BRDF (Eq. 1)
def ggx_D(cos_h, alpha):
    """GGX distribution (Walter et al. 2007), written with sin^2 to stay
    accurate for tiny alpha."""
    a2 = alpha * alpha
    c2 = cos_h * cos_h
    den = (1.0 - c2) + a2 * c2
    return np.where(cos_h > 0, a2 / (np.pi * den * den), 0.0)


def smith_G1(mu, alpha):
    a2 = alpha * alpha
    return np.where(mu > 0, 2.0 * mu / (mu + np.sqrt(a2 + (1.0 - a2) * mu * mu)), 0.0)


def spec_integrands(wi, wo, n, alpha):
    """F0*D*G/(4 n.wo) and F1*D*G/(4 n.wo) of Eq. 6 with the Fresnel split of
    Eq. 7, evaluated directly at incoming directions wi."""
    h = wi + wo
    h = h / np.linalg.norm(h, axis=-1, keepdims=True)
    mu_i = wi @ n
    mu_o = wo @ n
    c = np.sum(wi * h, axis=-1)
    F1 = (1.0 - c) ** 5
    F0 = 1.0 - F1
    base = ggx_D(h @ n, alpha) * smith_G1(mu_i, alpha) * smith_G1(mu_o, alpha) / (4.0 * mu_o)
    base = np.where((mu_i > 0) & (c > 0), base, 0.0)
    return F0 * base, F1 * base


def hemisphere_nodes(n_theta, n_phi):
    """Gauss-Legendre product rule on theta in [0, pi/2], phi in [0, 2 pi]:
    local directions and weights (including sin theta)."""
    xt, wt = leggauss(n_theta)
    xp, wp = leggauss(n_phi)
    th = 0.25 * np.pi * (xt + 1.0)
    ph = np.pi * (xp + 1.0)
    W = (0.25 * np.pi * wt)[:, None] * (np.pi * wp)[None, :] * np.sin(th)[:, None]
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    return d.reshape(-1, 3), W.ravel()


def half_vector_nodes(alpha, n_psi, n_phi):
    """Half vectors h(psi, phi) with tan(theta_h) = alpha * tan(psi), which
    concentrates nodes where D is large; weights = dOmega_h (explicit
    Jacobian sin(theta) d(theta)/d(psi))."""
    xs, ws = leggauss(n_psi)
    xp, wp = leggauss(n_phi)
    psi = 0.25 * np.pi * (xs + 1.0)
    ph = np.pi * (xp + 1.0)
    th = np.arctan(alpha * np.tan(psi))
    dth = alpha / np.cos(psi) ** 2 / (1.0 + (alpha * np.tan(psi)) ** 2)
    W = (0.25 * np.pi * ws * np.sin(th) * dth)[:, None] * (np.pi * wp)[None, :]
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    h = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    return h.reshape(-1, 3), W.ravel()


def white_furnace_AB(mu_o, alpha, n_psi, n_phi):
    """A = int F0 D G / (4 mu_o) d wi and B likewise with F1, integrated over
    half vectors: d wi = 4 (wo.h) d h."""
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([np.sqrt(1.0 - mu_o ** 2), 0.0, mu_o])
    h, W = half_vector_nodes(alpha, n_psi, n_phi)
    c = h @ wo
    wi = 2.0 * c[:, None] * h - wo
    f0, f1 = spec_integrands(wi, wo, n, alpha)
    jac = 4.0 * np.maximum(c, 0.0)
    return float(np.sum(f0 * jac * W)), float(np.sum(f1 * jac * W))


def white_furnace_AB_direct(mu_o, alpha, n):
    """Same integrals over incoming directions directly (no half vectors)."""
    nn = np.array([0.0, 0.0, 1.0])
    wo = np.array([np.sqrt(1.0 - mu_o ** 2), 0.0, mu_o])
    wi, W = hemisphere_nodes(n, 2 * n)
    f0, f1 = spec_integrands(wi, wo, nn, alpha)
    return float(np.sum(f0 * W)), float(np.sum(f1 * W))


# ----------------------------------------------------------------- helpers
def batch_bake(scene, q, batches, spp, spp_s=None, sigma=SIGMA):
    """Mean and standard error over independent request streams."""
    outs = [scene.bake(q, sigma, spp, spp_s, seed=1234, request_id=b)["flat"]
            for b in range(batches)]
    a = np.stack(outs)
    return a.mean(0), a.std(0, ddof=1) / np.sqrt(batches)


def one_query(x, n, wo, tri=-1):
    return {"x": np.array([x], np.float32), "n": np.array([n], np.float32),
            "wo": np.array([wo], np.float32), "tri": np.array([tri], np.int32)}


# ----------------------------------------------------------------- pins
def test_ggx_projected_distribution_integrates_to_one():
    for s in SIGMA:
        alpha = s * s
        f = lambda th: 2 * np.pi * ggx_D(np.cos(th), alpha) * np.cos(th) * np.sin(th)
        val, err = integrate.quad(f, 0, np.pi / 2, points=[alpha, 3 * alpha, 10 * alpha],
                                  limit=400, epsabs=1e-13, epsrel=1e-11)
        assert abs(val - 1.0) < 1e-8, (s, val)
        h, W = half_vector_nodes(alpha, 256, 16)
        assert abs(np.sum(ggx_D(h[:, 2], alpha) * h[:, 2] * W) - 1.0) < 1e-9


def test_half_vector_and_direct_quadratures_agree():
    for mu in (0.3, 1.0):
        for s in (0.5, 0.75, 1.0):
            a = white_furnace_AB(mu, s * s, 512, 512)
            b = white_furnace_AB_direct(mu, s * s, 512)
            assert np.allclose(a, b, rtol=2e-4, atol=1e-6), (mu, s, a, b)


def test_furnace_diffuse_is_exact():
    L = 0.7
    m = cornell_box(closed=True, furnace_radiance=L)
    S = O.OracleScene.from_mesh(m)
    q = surface_queries(m, 256, seed=5)
    r = S.bake(q, SIGMA, 32, 8)
    Lf = float(np.float32(L))
    assert np.max(np.abs(r["Ld"] - Lf)) < 1e-12


@pytest.mark.parametrize("mu_o", [0.05, 0.3, 0.7, 1.0])
def test_white_furnace_specular_matches_quadrature(mu_o):
    L = 1.0
    m = cornell_box(closed=True, furnace_radiance=L)
    S = O.OracleScene.from_mesh(m)
    wo = [np.sqrt(1.0 - mu_o ** 2), mu_o, 0.0]
    q = one_query([0.5, 0.0, 0.5], [0.0, 1.0, 0.0], wo)
    mean, se = batch_bake(S, q, 16, 4, 4096)
    K = len(SIGMA)
    for k, s in enumerate(SIGMA):
        A, B = white_furnace_AB(mu_o, s * s, 512, 256)
        A2, B2 = white_furnace_AB(mu_o, s * s, 1024, 512)
        qerr_a, qerr_b = abs(A - A2) + 1e-9, abs(B - B2) + 1e-9
        est_a = mean[0, 3 + 3 * k]
        est_b = mean[0, 3 + 3 * K + 3 * k]
        se_a = se[0, 3 + 3 * k]
        se_b = se[0, 3 + 3 * K + 3 * k]
        # 1e-6 absolute: GGX's long tail carries ~alpha^2 of the mass at
        # probabilities a 65536-sample run rarely visits, which the batch
        # standard error cannot see.  Likewise the samples whose reflected
        # direction falls below the horizon and count zero: a share q of at
        # most 1 - A - B, a handful of events in the run, so the bound adds
        # their binomial standard error sqrt(q / N) (stratified samples
        # leave little else for the batch error to show).
        N = 16 * 4096
        rare = np.sqrt(max(0.0, 1.0 - A2 - B2) / N)
        assert abs(est_a - L * A2) <= 4 * (se_a + rare) + qerr_a + 1e-6, (s, est_a, A2, se_a)
        assert abs(est_b - L * B2) <= 4 * (se_b + rare) + qerr_b + 1e-6, (s, est_b, B2, se_b)
        assert est_a + est_b <= 1.0 + 4 * (se_a + se_b) + 1e-7   # energy


def test_white_furnace_mirror_at_normal_incidence():
    # sigma -> 0 at wo = n: h = n, wo.h = 1, so F1 = 0 and G ~ 1.
    m = cornell_box(closed=True, furnace_radiance=1.0)
    S = O.OracleScene.from_mesh(m)
    r = S.bake(one_query([0.5, 0.0, 0.5], [0, 1, 0], [0, 1, 0]), [0.02], 4, 4096)
    assert r["Ls1"][0, 0, 0] < 1e-9
    assert abs(r["Ls0"][0, 0, 0] - 1.0) < 1e-5


def lambert_form_factor(x, n, poly):
    """Point-to-polygon form factor (Lambert): (1/2pi) sum_e angle_e * (n . g_e)."""
    tot = 0.0
    k = len(poly)
    for i in range(k):
        r0 = poly[i] - x
        r1 = poly[(i + 1) % k] - x
        g = np.cross(r0, r1)
        ang = np.arccos(np.clip(np.dot(r0, r1) / (np.linalg.norm(r0) * np.linalg.norm(r1)), -1, 1))
        tot += ang * np.dot(n, g / np.linalg.norm(g))
    return abs(tot) / (2 * np.pi)


@pytest.mark.parametrize("pt", [(0.5, 0.5), (0.2, 0.8), (0.9, 0.1)])
def test_emitter_form_factor_closed_form(pt):
    m = cornell_box(with_boxes=False, cache_value=0.0)
    S = O.OracleScene.from_mesh(m)
    x = np.array([pt[0], 0.0, pt[1]])
    q = one_query(x, [0, 1, 0], [0, 1, 0])
    mean, se = batch_bake(S, q, 16, 4096, 1, sigma=[0.5])
    ev = m.V[m.F[m.emitter]].reshape(-1, 3).astype(np.float64)
    y = ev[0, 1]
    poly = np.array([[0.35, y, 0.35], [0.65, y, 0.35], [0.65, y, 0.65], [0.35, y, 0.65]])
    # the origin is lifted by eps along n
    ff = lambert_form_factor(x + np.array([0, S.eps, 0]), np.array([0, 1.0, 0]), poly)
    Le = m.Le[m.emitter][0].astype(np.float64)
    for c in range(3):
        assert abs(mean[0, c] - Le[c] * ff) <= 4 * se[0, c] + 1e-9, (c, mean[0, c], Le[c] * ff)


def test_emission_is_one_sided():
    m = cornell_box(with_boxes=False, cache_value=0.0)
    S = O.OracleScene.from_mesh(m)
    # a ceiling point above the emitter only sees the emitter's back face
    q = one_query([0.5, 1.0, 0.5], [0, -1, 0], [0, -1, 0])
    r = S.bake(q, [0.5], 4096, 64)
    assert np.all(r["Ld"] == 0.0)
    # a floor point below it sees the front face (form factor ~0.03)
    q2 = one_query([0.5, 0.0, 0.5], [0, 1, 0], [0, 1, 0])
    assert np.all(S.bake(q2, [0.5], 4096, 1)["Ld"] > 0.1)


def hemisphere_quadrature(mesh, S, x, n, wo, alpha, nt, npz):
    """L_d and (L_s0, L_s1) at x by product quadrature over incoming
    directions; each node's ray is cast by brute force and its radiance is
    front-face emission + cache of the triangle it hits."""
    n = n / np.linalg.norm(n)
    t = np.cross(n, [1.0, 0, 0] if abs(n[0]) < 0.9 else [0, 1.0, 0])
    t /= np.linalg.norm(t)
    b = np.cross(n, t)
    dl, W = hemisphere_nodes(nt, npz)
    wi = dl[:, :1] * t + dl[:, 1:2] * b + dl[:, 2:] * n
    o = np.broadcast_to(x + S.eps * n, wi.shape)
    hit = S.closest(o, wi, brute=True)
    Li = np.zeros((len(wi), 3))
    ok = hit["id"] >= 0
    Li[ok] = mesh.cache[hit["id"][ok]] + hit["front"][ok, None] * mesh.Le[hit["id"][ok]]
    Ld = (Li * (dl[:, 2:] / np.pi) * W[:, None]).sum(0)
    f0, f1 = spec_integrands(wi, np.broadcast_to(wo, wi.shape), n, alpha)
    Ls0 = (Li * (f0 * W)[:, None]).sum(0)
    Ls1 = (Li * (f1 * W)[:, None]).sum(0)
    return Ld, Ls0, Ls1


@pytest.mark.parametrize("idx", [3, 17])
def test_cornell_point_matches_brute_force_hemisphere_quadrature(idx):
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    q = surface_queries(m, 32, seed=0)
    q1 = {k: v[idx:idx + 1] for k, v in q.items()}
    sig = 0.5
    mean, se = batch_bake(S, q1, 16, 4096, 4096, sigma=[sig])
    x, n, wo = (q1[k][0].astype(np.float64) for k in ("x", "n", "wo"))
    n = n / np.linalg.norm(n)
    wo = wo / np.linalg.norm(wo)
    hi = hemisphere_quadrature(m, S, x, n, wo, sig * sig, 256, 512)
    lo = hemisphere_quadrature(m, S, x, n, wo, sig * sig, 128, 256)
    for j, (a, b) in enumerate(zip(hi, lo)):
        est = mean[0, 3 * j:3 * j + 3]
        err = se[0, 3 * j:3 * j + 3]
        assert np.all(np.abs(est - a) <= 4 * err + 2 * np.abs(a - b) + 1e-6), (j, est, a, b, err)


@pytest.mark.parametrize("S", [1, 2, 7, 12, 16, 100, 128, 256, 4096])
def test_lobe_samples_are_jittered_strata(S):
    """A pair's S lobe samples cover an nx x ny grid over (u1, u2) with
    nx * ny = S, one sample per cell (nx the largest divisor of S with
    nx^2 <= S), each placed in its cell by its own uniforms, all in [0, 1)."""
    s = np.arange(S, dtype=np.uint32)
    c1, c2 = O.strat_uv(S, s, np.zeros(S), np.zeros(S))       # cell corners
    x1, x2 = np.unique(c1), np.unique(c2)
    nx, ny = len(x1), len(x2)
    assert nx * ny == S and nx <= ny and S % nx == 0
    assert all(S % d or d <= nx for d in range(1, int(np.sqrt(S)) + 1))  # nx the largest such divisor
    assert np.allclose(x1, np.arange(nx) / nx) and np.allclose(x2, np.arange(ny) / ny)
    cells = set(zip(np.rint(c1 * nx).astype(int), np.rint(c2 * ny).astype(int)))
    assert len(cells) == S                                       # every cell exactly once
    rng = np.random.default_rng(S)
    r1, r2 = rng.random(S), rng.random(S)
    r1[:2] = [0.0, 1.0 - 2.0 ** -24][:S]               # the extreme uniforms a Philox word gives
    r2[:2] = [1.0 - 2.0 ** -24, 0.0][:S]
    u1, u2 = O.strat_uv(S, s, r1, r2)
    assert np.all((u1 >= 0) & (u1 < 1) & (u2 >= 0) & (u2 < 1))
    # in its cell (float32 may round a sample at the cell's far edge onto the
    # next cell's boundary)
    assert np.all((u1 * nx >= np.rint(c1 * nx) - 1e-6) & (u1 * nx <= np.rint(c1 * nx) + 1 + 1e-6))
    assert np.all((u2 * ny >= np.rint(c2 * ny) - 1e-6) & (u2 * ny <= np.rint(c2 * ny) + 1 + 1e-6))
    assert np.allclose(u1 - c1, r1 / nx, rtol=0, atol=1e-6) and np.allclose(u2 - c2, r2 / ny, rtol=0, atol=1e-6)
    # formed in float32 (as the kernels form them): each value is a float32
    assert np.array_equal(u1, u1.astype(np.float32).astype(np.float64))


def test_stratified_estimate_keeps_its_mean_and_lowers_its_variance():
    """Over many independent pairs the stratified estimate of a smooth
    integral over [0,1)^2 has the integral's mean and a far smaller spread
    than independent samples."""
    S, pairs = 64, 2000
    rng = np.random.default_rng(3)
    f = lambda a, b: np.sin(3 * a) * (1 + b * b)
    exact = (1 - np.cos(3.0)) / 3 * (4.0 / 3)
    s = np.tile(np.arange(S, dtype=np.uint32), pairs)
    r1, r2 = rng.random(S * pairs), rng.random(S * pairs)
    u1, u2 = O.strat_uv(S, s, r1, r2)
    strat = f(u1, u2).reshape(pairs, S).mean(1)
    iid = f(r1, r2).reshape(pairs, S).mean(1)
    assert abs(strat.mean() - exact) < 4 * strat.std() / np.sqrt(pairs)
    assert strat.std() < 0.35 * iid.std()          # 0.24 measured; independent samples give 1
