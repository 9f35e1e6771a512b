"""Reciprocity pins for the oracle, CPU only.

* The BRDF of Eq. 1 (as the refinement evaluates it) is symmetric:
  f_r(wo, wi) = f_r(wi, wo) pointwise.  An asymmetric slip (G1(mu_o)^2
  for G1(mu_i) G1(mu_o), the Fresnel factor at wi.n instead of at the half
  vector) breaks it.
* Form factors obey A_i F_ij = A_j F_ji.  With L_e = 1 on patch j (cache 0
  everywhere) the bake's L_d at a point of patch i is the point-to-patch
  form factor, so averaging the oracle's L_d over uniform points of i
  estimates F_ij; swapping the emitting patch estimates F_ji.  This pins
  the sampling, the one-sided emission and the closest hit of the bake
  together, within Monte Carlo error."""
import numpy as np

import oracle as O
from workloads import cornell_box, surface_queries


def unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def test_brdf_is_reciprocal():
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(2000):
        n = unit(rng.normal(size=3))
        a, b = unit(rng.normal(size=3)), unit(rng.normal(size=3))
        a = a if a @ n > 0 else -a
        b = b if b @ n > 0 else -b
        if a @ n < 0.05 or b @ n < 0.05:
            continue
        alb = rng.uniform(0, 1, 3).astype(np.float32)
        sg, mt = float(rng.uniform(0.05, 1.0)), float(rng.uniform(0, 1))
        f_ab = O.brdf_cos(n, a, b, alb, sg, mt) / (n @ b)
        f_ba = O.brdf_cos(n, b, a, alb, sg, mt) / (n @ a)
        assert np.all(f_ab > 0)
        worst = max(worst, float(np.max(np.abs(f_ab - f_ba) / f_ab)))
    assert worst < 1e-12, worst


def patch_mean_Ld(m, Le, on_patch, N, S, seed):
    """Mean of the oracle's L_d over N area-uniform points of one patch."""
    over = 8
    while True:                      # area-uniform over the mesh, kept on the patch
        q = surface_queries(m, over * N, seed=seed, all_triangles=True)
        sel = np.nonzero(on_patch[q["tri"]])[0][:N]
        if len(sel) == N:
            break
        over *= 4
    qq = {key: v[sel] for key, v in q.items()}
    S_ = O.OracleScene(m.V, m.F, Le, np.zeros_like(m.Le))
    Ld = S_.bake(qq, [0.5], S, 1, seed=seed)["Ld"][:, 0]
    return Ld.mean(), Ld.std(ddof=1) / np.sqrt(N)


def tri_area(m, t):
    v = m.V[m.F[t]].astype(np.float64)
    return 0.5 * np.linalg.norm(np.cross(v[1] - v[0], v[2] - v[0]))


def test_form_factor_reciprocity_floor_and_light():
    m = cornell_box(with_boxes=False)
    floor, light = m.floor.copy(), m.emitter.copy()
    A_f = sum(tri_area(m, t) for t in np.nonzero(floor)[0])
    A_l = sum(tri_area(m, t) for t in np.nonzero(light)[0])
    Le = np.zeros_like(m.Le)
    Le[light] = 1.0
    F_fl, e_fl = patch_mean_Ld(m, Le, floor, 3000, 256, seed=1)
    Le = np.zeros_like(m.Le)
    Le[floor] = 1.0
    F_lf, e_lf = patch_mean_Ld(m, Le, light, 3000, 256, seed=2)
    lhs, rhs = A_f * F_fl, A_l * F_lf
    sig = np.hypot(A_f * e_fl, A_l * e_lf)
    # a 0.3 x 0.3 light 1 unit above a unit floor: F_floor->light ~ 0.02, F_light->floor ~ 0.24
    assert 0.01 < F_fl < 0.05 and 0.15 < F_lf < 0.35, (F_fl, F_lf)
    assert abs(lhs - rhs) < 4 * sig, (lhs, rhs, sig)
