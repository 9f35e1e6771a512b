"""fipt_render_fwd_noalloc: the render forward for callers that cannot
allocate device memory while they render (for example a service whose
device memory is a fixed pool sized at start-up, or a thread that must not
take an allocator's lock).
Its loss partial sums live in a fixed array inside the library instead of a
caller workspace.  Checked through the C ABI against the FP64 oracle's
render (Eq. 5, 8, 14) and against fipt_render_fwd, on two calls in a row
(the second call reuses the array the first one left behind), and at the
largest size the array allows.  This file is collected last so a
stop-at-first-failure run has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from workloads import material_params, shading_tables

pytestmark = pytest.mark.gpu

GRID = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
REL = 1e-4   # the render tests' tolerance
N_MAX = 131072 * 128         # FIPT_NOALLOC_RENDER_MAX_BLOCKS x 128 threads


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _host_inputs(N, seed):
    Ld, Ls0, Ls1 = shading_tables(N, len(GRID), seed=seed)
    mp = material_params(N, seed=seed + 1)
    gt = material_params(N, seed=seed + 2)
    Lgt = (Ld * gt["albedo"] + Ls0[:, 2] * 0.3).astype(np.float32)
    mask = (np.random.default_rng(seed).random(N) < 0.8).astype(np.uint8)
    return [Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask]


def _cuda(arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def _close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.maximum(np.abs(b), np.mean(np.abs(b)))
    assert np.max(np.abs(a - b) / scale) <= REL


def _noalloc(h, N):
    from paper_2304_05669_gb300._native import lib, check
    Ld, Ls0, Ls1, a, r, m, Lgt, mask = h
    grid = (ctypes.c_float * len(GRID))(*GRID)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Lr = torch.empty((N, 3), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    check(lib().fipt_render_fwd_noalloc(_p(Ld), _p(Ls0), _p(Ls1), N, len(GRID), grid, _p(a), _p(r),
                                        _p(m), _p(Lgt), _p(mask), _p(Lr), _p(loss), st))
    torch.cuda.synchronize()
    return Lr, loss


def test_noalloc_render_matches_oracle_and_workspace_render_twice():
    import paper_2304_05669_gb300 as F
    for N, seed in ((300001, 5), (4097, 9)):     # two calls in a row, different sizes
        host = _host_inputs(N, seed)
        d = _cuda(host)
        Lr, loss = _noalloc(d, N)
        Lr_ora, loss_ora = O.render_forward(*host[:3], GRID, *host[3:])
        _close(Lr.cpu().numpy(), Lr_ora)
        assert abs(loss.item() - loss_ora) <= REL * abs(loss_ora)
        Lr_ref, loss_ref = F.render_fwd(*d[:3], GRID, *d[3:])
        assert torch.equal(Lr, Lr_ref)
        assert abs(loss.item() - loss_ref.item()) <= REL * abs(loss_ref.item())


def test_noalloc_render_at_its_largest_size():
    """N = 16,777,216, the most the fixed array serves: 16 copies of one
    2^20-point input, so every copy's Lr must equal the first copy's bit for
    bit and the loss must be 16 times the oracle's loss of one copy."""
    base = 1 << 20
    host = _host_inputs(base, 21)
    reps = N_MAX // base
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda().repeat((reps,) + (1,) * (a.ndim - 1))
         for a in host]
    Lr, loss = _noalloc(d, N_MAX)
    Lr_ora, loss_ora = O.render_forward(*host[:3], GRID, *host[3:])
    first = Lr[:base]
    assert torch.equal(Lr.view(reps, base, 3), first.unsqueeze(0).expand(reps, base, 3))
    _close(first.cpu().numpy(), Lr_ora)
    assert abs(loss.item() - reps * loss_ora) <= REL * reps * abs(loss_ora)


def test_noalloc_render_rejects_sizes_beyond_its_scratch():
    from paper_2304_05669_gb300._native import lib
    L = lib()
    grid = (ctypes.c_float * len(GRID))(*GRID)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    N = N_MAX + 1
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.fipt_render_fwd_noalloc(_p(dummy), _p(dummy), _p(dummy), N, len(GRID), grid, _p(dummy),
                                   _p(dummy), _p(dummy), _p(dummy), None, _p(dummy), _p(loss), st)
    assert rc == 1
    assert b"exceeds its fixed scratch" in L.fipt_last_error()
