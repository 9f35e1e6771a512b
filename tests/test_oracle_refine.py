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
