"""GPU LBVH vs the oracle's bit-exact targets: Morton codes, sorted order,
radix-tree topology (as (first, last, split) triples) and node boxes."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import building_floor, cornell_box, procedural_room

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    assert torch.cuda.is_available()
    return F


def _compare(F, V, F_idx):
    T = len(F_idx)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Le = np.zeros((T, 3), np.float32)
    sc = F.Scene(t(V), t(F_idx), t(Le), t(Le), optimize=0)      # the radix tree as built
    ex = {k: v.cpu().numpy() for k, v in sc.export().items()}
    ref = O.lbvh_reference(V, F_idx)
    assert np.array_equal(ex["morton"].view(np.uint64), ref["sorted_codes"])
    assert np.array_equal(ex["order"], ref["order"])
    if T >= 2:
        g = {tuple(r): i for i, r in enumerate(ex["range"].tolist())}
        o = {(f, l, s): i for i, (f, l, s) in enumerate(zip(ref["first"].tolist(), ref["last"].tolist(),
                                                            ref["split"].tolist()))}
        assert set(g) == set(o)
        gi = np.array([g[k] for k in o])
        oi = np.array(list(o.values()))
        assert np.array_equal(ex["box"][gi], ref["node_box"][oi])
    F.context().sync_status()
    return sc


@pytest.mark.parametrize("name", ["cornell", "room", "random1000", "dups"])
def test_lbvh_bit_exact(fipt, name):
    rng = np.random.default_rng(11)
    if name == "cornell":
        m = cornell_box()
        V, Fi = m.V, m.F
    elif name == "room":
        m = procedural_room(1)
        V, Fi = m.V, m.F
    elif name == "random1000":
        V = rng.uniform(-3, 7, (3000, 3)).astype(np.float32)
        Fi = np.arange(3000, dtype=np.int32).reshape(1000, 3)
    else:  # many identical centres: ties broken by triangle index
        pts = rng.integers(0, 4, (500, 3)).astype(np.float32)
        V = np.repeat(pts, 3, axis=0)
        Fi = np.arange(1500, dtype=np.int32).reshape(500, 3)
    _compare(fipt, V, Fi)


def test_lbvh_bit_exact_two_million(fipt):
    m = building_floor(5)
    _compare(fipt, m.V, m.F)


@pytest.mark.parametrize("T", [1, 2, 3])
def test_lbvh_tiny_scenes(fipt, T):
    rng = np.random.default_rng(T)
    V = rng.uniform(0, 1, (3 * T, 3)).astype(np.float32)
    Fi = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    _compare(fipt, V, Fi)


def test_empty_scene_misses_everything(fipt):
    V = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    Fi = torch.zeros((0, 3), dtype=torch.int32, device="cuda")
    z = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    sc = fipt.Scene(V, Fi, z, z)
    o = torch.zeros((5, 3), device="cuda")
    d = torch.tensor([[0, 0, 1.0]] * 5, device="cuda")
    tri, t, fr = sc.trace(o, d)
    assert (tri.cpu() == -1).all() and torch.isinf(t.cpu()).all()
