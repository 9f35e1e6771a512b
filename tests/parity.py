"""Comparison rules shared by the GPU parity tests.

Bake tolerance (floating point).  The kernel accumulates float32 samples in
sample order and divides once; the oracle does the same in float64.  With
S <= 256 terms of magnitude <= max|L_i * w| the float32 sum is exact to
about S * 2^-24 relative to that magnitude, < 2e-5 for S = 256, and the
float32 sampling (directions, Fresnel, masking) perturbs each weight by a
few ulps.  The per-value bar is therefore
    |gpu - oracle| <= 1e-4 * max(|oracle|, mean over points of |oracle|)
(relative 1e-4, the mean floor keeping near-zero values from demanding
more than float32 can give).  Where a ray has several correct first hits
(see oracle/__init__.py), the oracle's [lo, hi] range replaces its value.
"""
import numpy as np

BAKE_REL = 1e-4
ETA_BAKE = 4e-6     # candidate-hit margin for rays the two sides generate independently
ETA_TRACE = 1e-6    # margin when both sides trace the same float32 ray


def bake_flat(Ld, Ls0, Ls1):
    N = Ld.shape[0]
    return np.concatenate([np.asarray(Ld).reshape(N, 3), np.asarray(Ls0).reshape(N, -1),
                           np.asarray(Ls1).reshape(N, -1)], axis=1).astype(np.float64)


def check_bake(gpu_flat, ora, rel=BAKE_REL, max_ambiguous_frac=None):
    """gpu_flat [N, 3+6K]; ora: oracle bake dict with lo/hi (eta > 0)."""
    nom, lo, hi = ora["flat"], ora["lo"], ora["hi"]
    scale = np.maximum(np.abs(nom), np.mean(np.abs(nom), axis=0, keepdims=True))
    tol = rel * scale
    below = gpu_flat < lo - tol
    above = gpu_flat > hi + tol
    bad = below | above
    exact = lo == hi
    err = np.abs(gpu_flat - nom) / np.where(scale > 0, scale, 1.0)
    rep = {"values": int(nom.size), "bad": int(bad.sum()),
           "unambiguous_frac": float(exact.mean()),
           "max_rel_err_unambiguous": float(err[exact].max()) if exact.any() else 0.0,
           "ambiguous_rays": int(ora["n_amb"].sum())}
    if bad.any():
        i, j = np.argwhere(bad)[0]
        rep["first_bad"] = (int(i), int(j), float(gpu_flat[i, j]), float(lo[i, j]),
                            float(nom[i, j]), float(hi[i, j]))
    assert not bad.any(), rep
    if max_ambiguous_frac is not None:
        assert 1.0 - rep["unambiguous_frac"] <= max_ambiguous_frac, rep
    return rep


def check_hits(g_tri, g_t, g_front, ora, t_rel=1e-5, L=1.0):
    """GPU closest hits against the oracle's candidate sets."""
    n = len(g_tri)
    amb = 0
    bad = []
    for r in range(n):
        nc = ora["n_cand"][r]
        cands = set(ora["cand_id"][r, :max(nc, 0)].tolist())
        if ora["miss_possible"][r]:
            cands.add(-1)
        if ora["id"][r] >= 0:
            cands.add(int(ora["id"][r]))
        else:
            cands.add(-1)
        if nc < 0:
            amb += 1
            continue
        if len(cands) > 1:
            amb += 1
        if int(g_tri[r]) not in cands:
            bad.append(r)
            continue
        if len(cands) == 1 and g_tri[r] >= 0:
            if abs(float(g_t[r]) - ora["t"][r]) > t_rel * (L + ora["t"][r]):
                bad.append(r)
            elif bool(g_front[r]) != bool(ora["front"][r]):
                bad.append(r)
    return amb, bad
