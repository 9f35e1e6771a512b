"""GPU sampler stream, closest hits, watertightness, camera first hits and
query compaction vs the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import ETA_TRACE, check_hits
from workloads import cornell_box, pinhole_views, procedural_room

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def test_philox_stream_matches_oracle(fipt):
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    g = fipt.philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                    torch.from_numpy(key.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(g, O.philox4x32_10(ctr, key))


def test_philox_matches_curand(fipt, tmp_path):
    """The library's Philox4x32-10 and the oracle's against CUDA's own
    (curand_Philox4x32_10, compiled here into a small test helper) on the
    same counters and keys."""
    import ctypes
    import os
    import subprocess
    from paper_2304_05669_gb300 import build as nb
    so = tmp_path / "libcurand_philox.so"
    subprocess.run([nb._nvcc(), *nb.ARCH, "-O2", "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
                    os.path.join(os.path.dirname(__file__), "c", "curand_philox.cu"), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    rng = np.random.default_rng(1)
    n = 1 << 18
    ctr = rng.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xffffffff] * 4, [1, 2, 3, 4], [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]]
    key[:4] = [[0, 0], [0xffffffff] * 2, [5, 6], [0xa4093822, 0x299f31d0]]
    ref = np.zeros((n, 4), np.uint32)
    P = ctypes.c_void_p
    assert L.curand_philox_batch(P(ctr.ctypes.data), P(key.ctypes.data), ctypes.c_int64(n), P(ref.ctypes.data)) == 0
    g = fipt.philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                    torch.from_numpy(key.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
    assert np.array_equal(g, ref)
    assert np.array_equal(O.philox4x32_10(ctr, key), ref)


def _rays(rng, lo, hi, n):
    o = rng.uniform(lo + 0.02, hi - 0.02, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d.astype(np.float32)


@pytest.mark.parametrize("scene", ["cornell", "room"])
def test_closest_hits_match_oracle(fipt, scene):
    m = cornell_box() if scene == "cornell" else procedural_room(1)
    sc = fipt.Scene.from_mesh(m)
    S = O.OracleScene.from_mesh(m)
    rng = np.random.default_rng(5)
    n = 200000 if scene == "cornell" else 100000
    o, d = _rays(rng, S.lo, S.hi, n)
    # a few axis-aligned and zero-component directions
    d[:6] = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float32)
    tri, t, fr = sc.trace(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    ora = S.closest(o.astype(np.float64), d.astype(np.float64), eta=ETA_TRACE)
    amb, bad = check_hits(tri.cpu().numpy(), t.cpu().numpy(), fr.cpu().numpy(), ora, L=S.L)
    assert bad == [], (len(bad), bad[:5])
    # ties and near-edge rays are rare
    assert amb / n < 0.02, amb / n
    fipt.context().sync_status()


def test_skip_triangle(fipt):
    m = cornell_box()
    sc = fipt.Scene.from_mesh(m)
    S = O.OracleScene.from_mesh(m)
    o = np.array([[0.5, 0.5, 0.5]], np.float32)
    d = np.array([[0.0, -1.0, 0.0]], np.float32)
    first = sc.trace(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())[0].item()
    skip = torch.tensor([first], dtype=torch.int32, device="cuda")
    second = sc.trace(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), skip)[0].item()
    ref = S.closest(o.astype(np.float64), d.astype(np.float64), skip=np.array([first], np.int32))
    assert second == ref["id"][0] and second != first


def test_closed_box_is_watertight(fipt):
    m = cornell_box(closed=True)
    sc = fipt.Scene.from_mesh(m)
    rng = np.random.default_rng(9)
    n = 1 << 20
    o = rng.uniform(0.001, 0.999, (n, 3)).astype(np.float32)
    d = rng.normal(size=(n, 3)).astype(np.float32)
    # aim a quarter of the rays exactly at mesh vertices and edge midpoints
    V = m.V[m.F].reshape(-1, 3)
    tgt = np.concatenate([V, 0.5 * (m.V[m.F[:, 0]] + m.V[m.F[:, 1]])])
    k = n // 4
    d[:k] = tgt[rng.integers(0, len(tgt), k)] - o[:k]
    tri, t, fr = sc.trace(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    assert int((tri < 0).sum()) == 0


def test_camera_queries_match_oracle(fipt):
    m = procedural_room(1)
    sc = fipt.Scene.from_mesh(m)
    S = O.OracleScene.from_mesh(m)
    cams = pinhole_views(m, 3, seed=2)
    W, H = 96, 64
    q, valid = sc.camera_queries(torch.from_numpy(cams).cuda(), W, H)
    q = q.cpu().numpy()
    valid = valid.cpu().numpy()
    P = len(valid)
    pix = np.arange(P)
    ora = S.camera_queries(cams, W, H, pix, eta=ETA_TRACE)
    gtri = q[:, 9].copy().view(np.int32)
    unique = (ora["n_cand"] <= 1) & ~ora["miss_possible"]
    assert unique.mean() > 0.97
    assert np.array_equal(gtri[unique], ora["tri"][unique])
    assert np.array_equal(valid[unique], (ora["tri"][unique] >= 0).astype(np.int32))
    u = unique & (gtri >= 0)
    scale = S.L
    assert np.max(np.abs(q[u, 0:3] - ora["x"][u])) < 2e-6 * scale * 4
    assert np.max(np.abs(q[u, 3:6] - ora["n"][u])) < 1e-5
    assert np.max(np.abs(q[u, 6:9] - ora["wo"][u])) < 1e-5
    for r in np.nonzero(~unique)[0]:
        cands = set(ora["cand_id"][r, :max(ora["n_cand"][r], 0)].tolist()) | {int(ora["tri"][r])}
        if ora["miss_possible"][r]:
            cands.add(-1)
        assert int(gtri[r]) in cands


def test_compaction_keeps_order(fipt):
    rng = np.random.default_rng(4)
    P = 100003
    q = rng.normal(size=(P, 10)).astype(np.float32)
    valid = (rng.random(P) < 0.7).astype(np.int32)
    for max_out in (0, 1, 5000, P):
        out, pix, n_out = fipt.compact_queries(torch.from_numpy(q).cuda(),
                                               torch.from_numpy(valid).cuda(), max_out)
        idx = np.nonzero(valid)[0][:max_out]
        assert int(n_out.item()) == len(idx)
        assert np.array_equal(pix.cpu().numpy()[:len(idx)], idx)
        assert np.array_equal(out.cpu().numpy()[:len(idx)], q[idx])
