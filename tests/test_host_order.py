"""The order the server gives a served bake's points, computed on the host
(fipt_debug_host_query_order): a permutation of [0, n) sorted stably by
the 30-bit Morton code of the positions in the box (1024 cells per axis),
checked against numpy's stable sort of codes built here from the box, for
sizes that run on one and on several threads.  No GPU needed."""
import ctypes

import numpy as np
import pytest

from paper_2304_05669_gb300._native import check, lib


def morton_codes(x, lo, hi):
    u = (x - lo) / (hi - lo)
    c = np.clip(np.nan_to_num(u * np.float32(1024), nan=0.0), 0, 1023).astype(np.int64)
    key = np.zeros(len(x), np.int64)
    for b in range(10):
        for a in range(3):
            key |= ((c[:, a] >> b) & 1) << (3 * b + a)
    return key


@pytest.mark.parametrize("n", [1, 2, 100, 65537, 300000])
def test_host_order_is_the_stable_morton_sort(n):
    rng = np.random.default_rng(n)
    q = np.zeros((n, 10), np.float32)
    x = rng.uniform(-2.0, 3.0, (n, 3)).astype(np.float32)
    x[: n // 3] = np.round(x[: n // 3], 1)              # many equal codes: stability matters
    if n > 10:
        x[5] = [-9.0, 9.0, np.nan]                      # outside the box and NaN clamp to the border cells
    q[:, 0:3] = x
    lo = np.array([-2.0, -2.0, -2.0], np.float32)
    hi = np.array([3.0, 3.0, 3.0], np.float32)
    out = np.empty(n, np.int32)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    check(lib().fipt_debug_host_query_order(p(q), n, p(lo), p(hi), p(out)))
    ref = np.argsort(morton_codes(x, lo, hi), kind="stable")
    assert np.array_equal(out, ref)
