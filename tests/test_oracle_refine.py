"""Pins for the oracle's stage-3 refinement (Sec. 4.3, Eq. 10; MIS per
Sec. 6), CPU only:
  * with MIS off and every surface rougher than the threshold, each sample
    is exactly the stage-1 bake's sample (same Philox stream, one segment);
  * with MIS on, the estimator has the same expectation as the stage-1
    bake (emitter sampling only re-weights how emitter light is found);
  * a near-mirror floor (sigma = 0.02, a = 1, m = 1, so F = 1) shows the
    emitter's mirror image: L_d at a ceiling point = L_e x Lambert's form
    factor of the reflected emitter polygon.
"""
import numpy as np
import pytest

import oracle as O
from test_oracle_bake import lambert_form_factor
from workloads import cornell_box, surface_queries

SIGMA = [0.02, 0.25, 1.0]


def mats(m, rough=1.0):
    T = m.T
    return (np.full((T, 3), 0.5, np.float32), np.full(T, rough, np.float32),
            np.zeros(T, np.float32))


def test_reduces_to_stage_one_without_mis_on_rough_scenes():
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    q = surface_queries(m, 200, seed=2)
    a, r, mt = mats(m, rough=1.0)
    ref = S.bake(q, SIGMA, 32, 16, seed=5, request_id=2)
    got = S.refine(q, SIGMA, 32, 16, a, r, mt, sigma_c=0.6, mis=False, seed=5, request_id=2)
    assert np.allclose(got["flat"], ref["flat"], rtol=1e-13, atol=1e-15)


def _specular_toward_emitter():
    """A floor point whose viewing direction mirrors the direction to the
    emitter's centre, so its glossy lobes see the emitter."""
    x = np.array([0.5, 0.0, 0.3])
    d = np.array([0.5, 0.999, 0.5]) - x
    d /= np.linalg.norm(d)
    wo = np.array([-d[0], d[1], -d[2]])
    return {"x": np.array([x], np.float32), "n": np.array([[0, 1, 0]], np.float32),
            "wo": np.array([wo], np.float32), "tri": np.array([-1], np.int32)}


@pytest.mark.parametrize("idx", [0, 7, -1])
def test_mis_keeps_the_expectation_of_stage_one(idx):
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    if idx < 0:
        q = _specular_toward_emitter()
    else:
        q = {k: v[idx:idx + 1] for k, v in surface_queries(m, 16, seed=3).items()}
    a, r, mt = mats(m, rough=1.0)
    outs_b, outs_r = [], []
    for b in range(12):
        outs_b.append(S.bake(q, SIGMA, 4096, 1024, seed=9, request_id=b)["flat"][0])
        outs_r.append(S.refine(q, SIGMA, 4096, 1024, a, r, mt, mis=True, seed=9,
                               request_id=b)["flat"][0])
    B, R = np.array(outs_b), np.array(outs_r)
    se = np.sqrt(B.var(0, ddof=1) / len(B) + R.var(0, ddof=1) / len(R))
    assert np.all(np.abs(B.mean(0) - R.mean(0)) <= 4 * se + 1e-6 * (1 + np.abs(B.mean(0))))
    # emitter sampling lowers the variance of the diffuse term under the light
    assert R[:, :3].var(0).sum() <= B[:, :3].var(0).sum() * 1.05


def test_mirror_floor_reflects_the_emitter():
    m = cornell_box(with_boxes=False, cache_value=0.0)
    S = O.OracleScene.from_mesh(m)
    T = m.T
    a = np.ones((T, 3), np.float32)
    r = np.ones(T, np.float32)
    mt = np.zeros(T, np.float32)
    floor = m.floor
    r[floor] = 0.02
    mt[floor] = 1.0
    x = np.array([0.15, 1.0, 0.15])
    q = {"x": np.array([x], np.float32), "n": np.array([[0, -1, 0]], np.float32),
         "wo": np.array([[0, -1, 0]], np.float32), "tri": np.array([-1], np.int32)}
    vals = [S.refine(q, [0.5], 16384, 1, a, r, mt, mis=True, seed=1, request_id=b)["flat"][0, :3]
            for b in range(48)]
    v = np.array(vals)
    ev = m.V[m.F[m.emitter]].reshape(-1, 3).astype(np.float64)
    y = -ev[0, 1]                                   # the emitter's image below the floor
    poly = np.array([[0.35, y, 0.35], [0.65, y, 0.35], [0.65, y, 0.65], [0.35, y, 0.65]])
    ff = lambert_form_factor(x - np.array([0, S.eps, 0]), np.array([0, -1.0, 0]), poly)
    Le = m.Le[m.emitter][0].astype(np.float64)
    se = v.std(0, ddof=1) / np.sqrt(len(v))
    # GGX at sigma = 0.02 is a mirror to ~1e-6 in energy; allow 2e-3 relative
    assert np.all(np.abs(v.mean(0) - Le * ff) <= 4 * se + 2e-3 * Le * ff), (v.mean(0), Le * ff)
    # without the floor's reflection (all rough, cache 0) the point stays dark
    dark = S.refine(q, [0.5], 1024, 1, a, np.ones(T, np.float32), mt, mis=True)["flat"][0, :3]
    assert np.all(dark == 0)


def _mirror_pair_scene(a_mirror):
    """Cornell box without boxes, cache 0: floor and ceiling are metallic
    GGX mirrors (sigma = 0.02 <= sigma_c, metallic 1, albedo a, so
    k_d = 0 and the reflectance is Schlick's a + (1 - a)(1 - cos)^5); the
    side walls are rough (sigma = 1 > sigma_c) and dark, so paths that meet
    them end with 0."""
    m = cornell_box(with_boxes=False, cache_value=0.0)
    T = m.T
    ys = m.V[m.F][:, :, 1]
    ceiling = (ys == 1.0).all(1) & ~m.emitter
    mirror = m.floor | ceiling
    assert mirror.sum() == 4
    a = np.ones((T, 3), np.float32)
    r = np.ones(T, np.float32)
    mt = np.zeros(T, np.float32)
    a[mirror] = a_mirror
    r[mirror] = 0.02
    mt[mirror] = 1.0
    # wind the mirrors to face out of the box: a path vertex must turn the
    # geometric normal toward the ray it arrives on
    m.F[mirror] = m.F[mirror][:, ::-1]
    return m, a, r, mt


def test_two_mirror_image_and_depth_cut():
    """Floor and ceiling mirrors facing each other under the Cornell light.
    A floor point at (0.1, 0, 0.1) sees the light directly and, through the
    ceiling then the floor mirror, the light's second image: unfolded, the
    quad at y = 2 + 0.999, same x/z footprint (for this point the cone to
    that image clears the real light and its first, back-facing image).  The
    image reaches L_d through a path whose vertices 1 and 2 are mirrors, so
    with max_depth = 1 it is cut and L_d = L_e F_direct (Lambert's closed
    form); with max_depth = 2 (4-mirror images still cut)
    L_d = L_e (F_direct + J), J = (1/pi) int_quad R(cos)^2 h^2 / r^4 dA with
    R the Schlick reflectance of each bounce at the ray's incidence angle
    (h / r), by 2-D quadrature.  The throughput product at depth 2 (R^2 with
    a = 0.5, not R), the depth cut, the skipped triangle and the origin
    offset at later vertices all enter this difference."""
    from scipy import integrate
    from test_oracle_bake import lambert_form_factor
    am = 0.5
    m, a, r, mt = _mirror_pair_scene(am)
    S = O.OracleScene.from_mesh(m)
    npts = 32
    x = np.array([0.1, 0.0, 0.1])
    q = {"x": np.tile(x.astype(np.float32), (npts, 1)), "n": np.tile(np.float32([0, 1, 0]), (npts, 1)),
         "wo": np.tile(np.float32([0, 1, 0]), (npts, 1)), "tri": np.full(npts, -1, np.int32)}
    Le = m.Le[m.emitter][0].astype(np.float64)
    p = x + np.array([0, S.eps, 0])
    y = 0.999
    poly = np.array([[0.35, y, 0.35], [0.65, y, 0.35], [0.65, y, 0.65], [0.35, y, 0.65]])
    f_direct = lambert_form_factor(p, np.array([0, 1.0, 0]), poly)

    def kern(Z, X):
        h = 2.0 + y - p[1]
        r2 = (X - p[0]) ** 2 + h ** 2 + (Z - p[2]) ** 2
        c = h / np.sqrt(r2)
        R = am + (1 - am) * (1 - c) ** 5
        return R * R * h * h / (np.pi * r2 * r2)
    J = integrate.dblquad(kern, 0.35, 0.65, 0.35, 0.65, epsabs=1e-13, epsrel=1e-11)[0]
    for depth, ref in ((1, Le * f_direct), (2, Le * (f_direct + J))):
        out = S.refine(q, [0.5], 65536, 1, a, r, mt, max_depth=depth, mis=True, seed=7,
                       request_id=depth)["flat"][:, :3]
        mean, se = out.mean(0), out.std(0, ddof=1) / np.sqrt(npts)
        # the GGX lobe at sigma = 0.02 is a mirror to ~1e-5 in energy
        assert np.all(np.abs(mean - ref) <= 4 * se + 2e-3 * Le * J), (depth, mean, ref, se, Le * J)


def test_vertex_brdf_directional_albedo():
    """The full BRDF of Eq. 1 that a path vertex samples and evaluates
    (k_d / pi + (k_s F0 + F1) D G / (4 mu_o mu_i), times mu_i), integrated
    over incoming directions, is the directional albedo
    k_d + k_s A(mu_o, sigma) + B(mu_o, sigma), with A and B the split-sum
    integrals of the Fresnel factors (computed independently by quadrature in
    the bake's pins).  Metallic 1 leaves only the specular part
    (a A + B): a Fresnel split F0 = 1 would add a B; metallic 0 on a rough
    surface gives a + 0.04 A + B."""
    from test_oracle_bake import half_vector_nodes, hemisphere_nodes, white_furnace_AB
    n = np.array([0.0, 0.0, 1.0])
    alb = np.float32([0.7, 0.4, 0.2])
    for mu_o, sg, mt in ((0.3, 0.5, 1.0), (0.8, 0.3, 1.0), (0.5, 1.0, 0.0)):
        al = sg * sg
        wo = np.array([np.sqrt(1 - mu_o ** 2), 0.0, mu_o])
        A, B = white_furnace_AB(mu_o, al, 256, 256)
        if mt == 1.0:      # half-vector nodes follow the specular peak
            h, W = half_vector_nodes(al, 160, 160)
            c = h @ wo
            wi = 2.0 * c[:, None] * h - wo
            W = W * 4.0 * np.maximum(c, 0.0)
        else:              # a broad lobe: plain hemisphere nodes
            wi, W = hemisphere_nodes(160, 160)
        keep = (wi @ n > 0) & (W > 0)
        tot = np.zeros(3)
        for d, w in zip(wi[keep], W[keep]):
            tot += w * O.brdf_cos(n, wo, d, alb, sg, mt)
        kd = alb * (1 - mt)
        ks = 0.04 * (1 - mt) + alb * mt
        ref = kd + ks * A + B
        assert np.allclose(tot, ref, rtol=2e-5, atol=0), (mu_o, sg, mt, tot, ref)


def _perturb(q, seed):
    """The query records moved by 1-3 float32 ulps per component."""
    rng = np.random.default_rng(seed)
    out = dict(q)
    for k in ("x", "n", "wo"):
        v = np.array(q[k], np.float32)
        for _ in range(3):
            step = rng.integers(-1, 2, v.shape)
            v = np.where(step > 0, np.nextafter(v, np.float32(np.inf)),
                         np.where(step < 0, np.nextafter(v, np.float32(-np.inf)), v)).astype(np.float32)
        out[k] = v
    return out


def test_sample_ranges_bound_the_nominal_and_perturbed_paths():
    """The per-sample ranges (every decision a float32 path's accumulated
    rounding may flip) contain the nominal value and the values of the same
    samples computed from query records moved by a few float32 ulps, whose
    FP64 paths take some of those decisions the other way and drift
    continuously.  Room with random per-triangle materials (many glossy
    vertices, max_depth 8): few samples become unbounded.  Glossy Cornell
    walls with paths up to 40 vertices: the rounding of a hit point grows by
    about 1/cos per bounce, so a sizeable share of the deep samples lose
    track of their FP64 twin and are unbounded."""
    from workloads import procedural_room
    rng = np.random.default_rng(8)
    cases = []
    m = procedural_room(1)
    T = m.T
    cases.append((m, rng.uniform(0, 1, (T, 3)).astype(np.float32),
                  rng.uniform(0.02, 1.0, T).astype(np.float32),
                  rng.uniform(0, 1, T).astype(np.float32), surface_queries(m, 96, seed=6), 8, 8, 0.03))
    m2 = cornell_box()
    T2 = m2.T
    cases.append((m2, np.full((T2, 3), 0.8, np.float32), np.full(T2, 0.3, np.float32),
                  np.zeros(T2, np.float32), surface_queries(m2, 48, seed=22), 4, 40, 0.4))
    moved = 0
    for m, a, r, mt, q, spp, depth, max_unb in cases:
        S = O.OracleScene.from_mesh(m)
        o = S.refine(q, SIGMA, spp, spp, a, r, mt, max_depth=depth, eta=1e-5, per_sample=True,
                     bounds=True, seed=3, request_id=1)
        ps, lo, hi, unb = o["per_sample"], o["lo"], o["hi"], o["unbounded"]
        assert np.all(lo <= ps) and np.all(ps <= hi)
        assert unb.mean() <= max_unb, unb.mean()
        col = np.mean(np.abs(ps), axis=(0, 2), keepdims=True)
        tol = 1e-4 * np.maximum(np.abs(ps), col)
        for k in range(4):
            p = S.refine(_perturb(q, 100 + k), SIGMA, spp, spp, a, r, mt, max_depth=depth,
                         per_sample=True, seed=3, request_id=1)["per_sample"]
            out = ((p < lo - tol) | (p > hi + tol)) & ~unb[..., None]
            assert not out.any(), np.argwhere(out)[:5]
            moved += int(np.sum((np.abs(p - ps) > tol) & ~unb[..., None]))
    assert moved > 0            # some bounded samples did take another branch
