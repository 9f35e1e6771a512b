"""The emitter sampler splits a sample index i into (triangle, sample) by
dividing by the invariant samples-per-triangle n with one multiply-high
(Granlund and Montgomery 1994).  The library's own routine, run on the host
(no GPU needed) and in a kernel, must equal integer division for every
32-bit i; checked at the edges where such a routine can go wrong: n = 1
(no shift), powers of two (magic m = 1), divisors near 2^31 and 2^32, and
for every divisor the indices around each multiple of n near 0 and near
2^32 - 1, plus random indices."""
import ctypes

import numpy as np
import pytest


def divisors():
    ds = set(range(1, 2049)) | {1 << k for k in range(32)} | {(1 << k) + d for k in range(2, 32) for d in (-1, 1)}
    ds |= {1000, 100, 3, 7, 0x7FFFFFFF, 0xFFFFFFFF, 0xFFFFFFFE, 0x80000001, 641, 6700417}
    return sorted(d for d in ds if 1 <= d <= 0xFFFFFFFF)


def indices(n, rng):
    top = 0xFFFFFFFF
    i = [0, 1, 2, n - 1, n, n + 1, 2 * n - 1, 2 * n, top, top - 1, top - n, top - n + 1]
    q = top // n                          # the last multiples of n below 2^32
    for k in (q, q - 1):
        for d in (-1, 0, 1):
            i.append(k * n + d)
    i.extend(rng.integers(0, 1 << 32, 64, dtype=np.uint64).tolist())
    return np.array([v for v in i if 0 <= v <= top], dtype=np.uint32)


def _lib():
    from paper_2304_05669_gb300._native import lib
    return lib()


def test_host_division_matches_integer_division():
    L = _lib()
    rng = np.random.default_rng(1)
    for n in divisors():
        i = indices(n, rng)
        out = np.empty_like(i)
        rc = L.fipt_debug_divide(n, ctypes.c_void_p(i.ctypes.data), len(i), ctypes.c_void_p(out.ctypes.data),
                                 0, None)
        assert rc == 0
        ref = (i.astype(np.uint64) // np.uint64(n)).astype(np.uint32)
        assert np.array_equal(out, ref), (n, i[out != ref][:4])


@pytest.mark.gpu
def test_device_division_matches_integer_division():
    import torch
    L = _lib()
    rng = np.random.default_rng(2)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in divisors()[::7] + [1, 2, 7, 64, 1000]:
        i = indices(n, rng)
        d_i = torch.from_numpy(i.view(np.int32).copy()).cuda()
        d_o = torch.empty_like(d_i)
        assert L.fipt_debug_divide(n, ctypes.c_void_p(d_i.data_ptr()), len(i),
                                   ctypes.c_void_p(d_o.data_ptr()), 1, st) == 0
        out = d_o.cpu().numpy().view(np.uint32)
        ref = (i.astype(np.uint64) // np.uint64(n)).astype(np.uint32)
        assert np.array_equal(out, ref), (n, i[out != ref][:4])
