"""Pins for the oracle's Philox stream and LBVH targets (CPU only).

Philox4x32-10 is pinned to the published Random123 known-answer vectors.
Morton codes are pinned to hand-placed triangle centres, and the radix
tree to a brute-force construction from its definition (the compressed
binary trie of the augmented keys).
"""
import numpy as np
import pytest

import oracle as O
from conftest import read_golden
from workloads import cornell_box, procedural_room


def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(v[0:4], v[4:6])[0]
        assert [int(x) for x in out] == v[6:10]


def test_uniforms_are_exact_24_bit_fractions():
    w = np.array([0, 255, 256, 0xFFFFFFFF, 0x80000000], np.uint32)
    u = O.uniforms24(w)
    assert u.tolist() == [0.0, 0.0, 2.0 ** -24, 1.0 - 2.0 ** -24, 0.5]


def test_philox_streams_differ_per_counter_word():
    base = np.array([[5, 7, 1, 0]], np.uint32)
    outs = {tuple(O.philox4x32_10(base + np.eye(4, dtype=np.uint32)[i], [[9, 0]])[0])
            for i in range(4)}
    assert len(outs) == 4


def _point_tris(centres, lo=(0, 0, 0), hi=(1, 1, 1)):
    """Degenerate triangles whose box is a single point, plus two triangles
    pinning the scene box to [lo, hi]."""
    V, F = [], []
    for c in list(centres) + [lo, hi]:
        b = len(V)
        V += [c, c, c]
        F.append([b, b + 1, b + 2])
    return np.array(V, np.float32), np.array(F, np.int32)


def test_morton_hand_placed_centres():
    V, F = _point_tris([(1, 1, 1), (0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0, 0),
                        (0.25, 0.75, 0.125)])
    c = O.morton_codes(V, F)
    assert int(c[0]) == (1 << 63) - 1          # clamped to 2^21 - 1 on every axis
    assert int(c[1]) == 1 << 62                # qx = 2^20 -> bit 3*20 + 2
    assert int(c[2]) == 1 << 61                # qy = 2^20 -> bit 3*20 + 1
    assert int(c[3]) == 1 << 60                # qz = 2^20 -> bit 3*20
    assert int(c[4]) == 0
    # qx = 2^19, qy = 2^20 + 2^19, qz = 2^18
    assert int(c[5]) == (1 << 59) | (1 << 61) | (1 << 58) | (1 << 54)


def test_morton_cell_boundaries_round_down():
    # centre one float ulp below a cell boundary falls in the lower cell
    below = np.nextafter(np.float32(0.5), np.float32(0))
    V, F = _point_tris([(below, 0, 0), (0.5, 0, 0)])
    c = O.morton_codes(V, F)
    qx_below = int(np.floor(float(below) * 2 ** 21))
    assert qx_below == 2 ** 20 - 1
    spread = sum(((qx_below >> i) & 1) << (3 * i + 2) for i in range(21))
    assert int(c[0]) == spread and int(c[1]) == 1 << 62


def test_morton_flat_axis_quantises_to_zero():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [1, 0, 1]], np.float32)
    F = np.array([[0, 1, 2], [1, 3, 2]], np.int32)
    c = O.morton_codes(V, F)
    for code in c:                              # y bits (3i+1) all zero
        assert all(((int(code) >> (3 * i + 1)) & 1) == 0 for i in range(21))


def _brute_radix_tree(codes):
    """Internal nodes of the compressed binary trie of the keys (code || i)."""
    T = len(codes)
    keys = [(int(c) << 32) | i for i, c in enumerate(codes)]
    nodes = set()
    for level in range(96):
        start = 0
        while start < T:
            end = start
            pre = keys[start] >> (96 - level) if level else 0
            while end + 1 < T and ((keys[end + 1] >> (96 - level)) if level else 0) == pre:
                end += 1
            bits = [(keys[k] >> (95 - level)) & 1 for k in range(start, end + 1)]
            if end > start and 0 in bits and 1 in bits:
                split = start + bits.count(0) - 1
                nodes.add((start, end, split))
            start = end + 1
    return nodes


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radix_tree_matches_trie_definition(seed):
    rng = np.random.default_rng(seed)
    T = 150
    pts = rng.integers(0, 6, (T, 3)).astype(np.float32) / 5.0  # many duplicate codes
    V = np.repeat(pts, 3, axis=0)
    F = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    ref = O.lbvh_reference(V, F)
    got = set(zip(ref["first"].tolist(), ref["last"].tolist(), ref["split"].tolist()))
    assert len(got) == T - 1
    assert got == _brute_radix_tree(ref["sorted_codes"])


def test_radix_tree_invariants_on_room():
    m = procedural_room(1)
    ref = O.lbvh_reference(m.V, m.F)
    T = m.T
    f, l, s = ref["first"], ref["last"], ref["split"]
    assert len(f) == T - 1
    assert f[0] == 0 and l[0] == T - 1
    assert np.all((f <= s) & (s < l))
    # every child range is either a leaf or another node's range
    ranges = set(zip(f.tolist(), l.tolist()))
    for a, b, c in zip(f.tolist(), l.tolist(), s.tolist()):
        assert a == c or (a, c) in ranges
        assert c + 1 == b or (c + 1, b) in ranges
    # node boxes are the min / max over their triangles
    tb = ref["tri_box"]
    for k in np.random.default_rng(0).integers(0, T - 1, 200):
        box = ref["node_box"][k]
        assert np.array_equal(box[:3], tb[f[k]:l[k] + 1, :3].min(0))
        assert np.array_equal(box[3:], tb[f[k]:l[k] + 1, 3:].max(0))
    # the order is the stable (code, index) sort
    sc = ref["sorted_codes"]
    assert np.all(sc[:-1] <= sc[1:])
    eq = sc[:-1] == sc[1:]
    assert np.all(ref["order"][:-1][eq] < ref["order"][1:][eq])


def test_bvh_closest_equals_brute_force():
    rng = np.random.default_rng(0)
    for mesh, n in ((cornell_box(), 4000), (procedural_room(1), 300)):
        S = O.OracleScene.from_mesh(mesh)
        o = rng.uniform(S.lo + 0.05, S.hi - 0.05, (n, 3))
        d = rng.normal(size=(n, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        a = S.closest(o, d)
        b = S.closest(o, d, brute=True)
        assert np.array_equal(a["id"], b["id"])
        hit = a["id"] >= 0
        assert np.array_equal(a["t"][hit], b["t"][hit])
        assert np.array_equal(a["front"], b["front"])


def test_closest_hit_on_axis_aligned_wall():
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    o = np.array([[0.2, 0.9, 0.3]])
    r = S.closest(o, np.array([[1.0, 0.0, 0.0]]))
    assert r["t"][0] == pytest.approx(0.8, abs=1e-12)
    tri = r["id"][0]
    v = m.V[m.F[tri]]
    assert np.allclose(v[:, 0], 1.0)            # the x = 1 wall
    assert r["front"][0]                        # walls face into the room


def test_candidate_set_contains_both_sides_of_a_shared_edge():
    m = cornell_box()
    S = O.OracleScene.from_mesh(m)
    # back wall z=1 is split along a diagonal of the unit square; aim at it
    o = np.array([[0.7, 0.7, 0.5]])
    target = np.array([0.5, 0.5, 1.0])
    d = (target - o) / np.linalg.norm(target - o)
    r = S.closest(o, d, eta=1e-6)
    assert r["n_cand"][0] == 2
    back = [k for k in range(m.T) if np.allclose(m.V[m.F[k], 2], 1.0)]
    assert set(r["cand_id"][0, :2].tolist()) == set(back)
