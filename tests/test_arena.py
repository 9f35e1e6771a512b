"""Host-side admission bookkeeping of the serving runtime (fipt_arena_*),
checked against a plain Python interval model.  CPU only."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2304_05669_gb300 import _native
    return _native.lib()


def up(x):
    return (max(x, 1) + 255) // 256 * 256


def test_arena_matches_interval_model(L):
    size = 1 << 20
    a = ctypes.c_void_p()
    assert L.fipt_arena_create(size, ctypes.byref(a)) == 0
    rng = np.random.default_rng(0)
    live = {}
    for _ in range(4000):
        if live and rng.random() < 0.45:
            off = int(rng.choice(list(live)))
            assert L.fipt_arena_free(a, off, live.pop(off)) == 0
        else:
            want = int(rng.integers(1, 60000))
            off = ctypes.c_size_t()
            rc = L.fipt_arena_alloc(a, want, ctypes.byref(off))
            # first fit over the model's free gaps
            spans = sorted((o, up(b)) for o, b in live.items())
            gaps, cur = [], 0
            for o, b in spans:
                if o > cur:
                    gaps.append((cur, o - cur))
                cur = o + b
            if cur < size:
                gaps.append((cur, size - cur))
            fit = [g for g in gaps if g[1] >= up(want)]
            if fit:
                assert rc == 0 and off.value == fit[0][0]
                live[off.value] = want
            else:
                assert rc == 4          # FIPT_ERR_BUDGET
        used = ctypes.c_size_t()
        assert L.fipt_arena_info(a, ctypes.byref(used), None, None) == 0
        assert used.value == sum(up(b) for b in live.values())
    for off, b in list(live.items()):
        assert L.fipt_arena_free(a, off, b) == 0
    largest = ctypes.c_size_t()
    L.fipt_arena_info(a, None, None, ctypes.byref(largest))
    assert largest.value == size                 # everything coalesced back
    L.fipt_arena_destroy(a)


def test_arena_rejects_bad_frees(L):
    a = ctypes.c_void_p()
    L.fipt_arena_create(4096, ctypes.byref(a))
    off = ctypes.c_size_t()
    assert L.fipt_arena_alloc(a, 1000, ctypes.byref(off)) == 0
    assert L.fipt_arena_free(a, off.value + 1024, 256) == 1   # not allocated
    assert L.fipt_arena_free(a, off.value, 1000) == 0
    assert L.fipt_arena_free(a, off.value, 1000) == 1         # double free
    assert L.fipt_arena_alloc(a, 5000, ctypes.byref(off)) == 4
    L.fipt_arena_destroy(a)
