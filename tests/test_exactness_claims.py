"""CPU checks of the two exactness arguments the voxel pooling and the
emitter classification rest on (no GPU, no oracle):

1. n float32 values whose nonzero exponents span emax - emin <= 29 - bitlen(n)
   have an in-order FP64 sum equal to their exact sum, which is an integer
   multiple of 2^(emin - 150) below 2^53 units -- so an int64 sum in those
   units (in any order) reproduces the FP64 sum bit for bit.
2. The cell floor(RN64(RN64(x - lo) * scale)), clamped to [0, R - 1], equals
   the clamped floor of the float32 estimate RN32(RN32(x - lo) * RN32(scale))
   whenever no inner cell face (an integer in [1, R - 1]) lies within
   2^-21 |f| of the estimate f; only the pixels near a face need FP64.
"""
from fractions import Fraction

import numpy as np


def _exp_field(v):
    return (np.asarray(v, np.float32).view(np.uint32) >> 23) & 0xFF


def _spread_limit(n):
    return 29 - int(n).bit_length()


def _in_range(vals):
    nz = vals[vals != 0]
    if nz.size == 0:
        return True
    e = _exp_field(nz).astype(int)
    return e.min() >= 1 and e.max() < 255 and e.max() - e.min() <= _spread_limit(len(vals))


def test_inorder_fp64_sum_is_exact_in_range():
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(4000):
        n = int(rng.integers(1, 400))
        spread = max(_spread_limit(n), 0)
        e = rng.integers(-spread // 2, spread // 2 + 1, n)
        v = (rng.uniform(0.5, 1.0, n) * rng.choice([1.0, -1.0], n) * 2.0 ** e).astype(np.float32)
        v[rng.uniform(size=n) < 0.1] = 0.0
        if not _in_range(v):
            continue
        checked += 1
        s = 0.0
        for x in v:
            s += float(x)
        exact = sum((Fraction(float(x)) for x in v), Fraction(0))
        assert Fraction(s) == exact
        nz = v[v != 0]
        if nz.size:
            emin = int(_exp_field(nz).min())
            units = exact / Fraction(2) ** (emin - 150)
            assert units.denominator == 1 and abs(units.numerator) < 2 ** 53
    assert checked > 3000


def test_outside_the_range_fp64_can_round():
    # The bound is sufficient, not necessary: 1, 1.5 and 2^-29 fall outside
    # it (their sum needs 2^53 units of 2^-52) and still add exactly ...
    v = np.array([1.0, 1.5, 2.0 ** -29], np.float32)
    assert not _in_range(v)
    s = 0.0
    for x in v:
        s += float(x)
    assert s == 2.5 + 2.0 ** -29
    # ... but outside it FP64 additions can round: 2^-30 is half an ulp of
    # 2^24 - 1 in FP64 and ties to even, so both small terms are lost
    w = np.array([2.0 ** 24 - 1, 2.0 ** -30, 2.0 ** -30], np.float32)
    assert not _in_range(w)
    t = 0.0
    for x in w:
        t += float(x)
    assert Fraction(t) != sum((Fraction(float(x)) for x in w), Fraction(0))


def test_float32_cell_matches_fp64_away_from_faces():
    rng = np.random.default_rng(12)
    for R in (1, 7, 256, 1024):
        for lo_, hi_ in (((-0.1, -0.1, -0.1), (4.1, 3.1, 6.1)), ((-1e3, 5.0, 1e-3), (1e3, 7.5, 2e-3))):
            lo, hi = np.array(lo_, np.float32), np.array(hi_, np.float32)
            scale = R / (hi.astype(np.float64) - lo.astype(np.float64))
            n = 200000
            k = rng.integers(-2, R + 3, (n, 3))
            x = (lo.astype(np.float64) + k * (hi.astype(np.float64) - lo) / R).astype(np.float32)
            for _ in range(3):                               # walk a few ulps off the faces
                sel = rng.random((n, 3)) < 0.3
                towards = np.where(rng.random((n, 3)) < 0.5, np.float32(-np.inf), np.float32(np.inf))
                x = np.where(sel, np.nextafter(x, towards), x)
            x = np.concatenate([x, rng.uniform(lo - (hi - lo), hi + (hi - lo), (n, 3)).astype(np.float32)])
            with np.errstate(all="ignore"):
                f = (x - lo) * scale.astype(np.float32)       # float32 throughout
                r = np.rint(f)
                near = (r >= 1) & (r <= R - 1) & (np.abs(f - r) <= np.abs(f) * np.float32(2.0 ** -21))
                fast = np.clip(np.floor(f), 0, R - 1)
                ref = np.clip(np.floor((x.astype(np.float64) - lo.astype(np.float64)) * scale), 0, R - 1)
            taken = ~near
            assert np.array_equal(fast[taken], ref[taken])
            if R > 1:
                assert near.any()                            # the faces were reached
