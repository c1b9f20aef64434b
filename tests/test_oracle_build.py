"""Pins of the oracle's octree build against hand-checked cases and brute force (no GPU).

The build follows the PlenOctree structure the paper starts from (Sec. 3, Preliminaries): a cube
root subdivided 8-way (M = 8, Eq. 3), with the scene's cells refined to the maximum depth.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

Q = si.Q


def _decode(key):
    key = int(key)
    l = (key.bit_length() - 1) // 3
    k = [0, 0, 0]
    for i in range(l - 1, -1, -1):
        tri = (key >> (3 * i)) & 7
        k[0] = (k[0] << 1) | ((tri >> 2) & 1)
        k[1] = (k[1] << 1) | ((tri >> 1) & 1)
        k[2] = (k[2] << 1) | (tri & 1)
    return l, k


def _meets_bruteforce(prims, l, kx, ky, kz):
    """Cell-versus-primitive tests written another way: sphere by the clamped nearest point,
    boxes and cylinders by integer ranges of cells covering the open primitive."""
    sz = 1 << (24 - l)
    A = np.stack([kx * sz, ky * sz, kz * sz], axis=-1).astype(np.int64)
    B = A + sz
    hit = np.zeros(kx.shape, bool)
    for p in prims:
        t = int(p[0])
        q = [int(x) for x in p[1:]]
        if t == si.PRIM_SPHERE:
            c = np.array(q[:3], np.int64)
            near = np.clip(c, A, B)
            hit |= ((near - c) ** 2).sum(-1) < q[3] * q[3]
        elif t == si.PRIM_BOX:
            ok = np.ones(kx.shape, bool)
            for a in range(3):
                # cells whose open interval meets (lo, hi): floor(lo/sz) <= k <= ceil(hi/sz) - 1
                lo_c = q[a] // sz
                hi_c = -((-q[3 + a]) // sz) - 1
                kk = A[..., a] // sz
                ok &= (kk >= lo_c) & (kk <= hi_c)
            hit |= ok
        else:
            c = np.array([q[0], q[1]], np.int64)
            near = np.clip(c, A[..., [0, 2]], B[..., [0, 2]])
            disk = ((near - c) ** 2).sum(-1) < q[2] * q[2]
            lo_c = q[3] // sz
            hi_c = -((-q[4]) // sz) - 1
            ky_ = A[..., 1] // sz
            hit |= disk & (ky_ >= lo_c) & (ky_ <= hi_c)
    return hit


def test_depth1_single_sphere_by_hand():
    # sphere at normalised (0.25, 0.25, 0.25), radius 0.1: only octant 0 meets it
    prims = np.array([[si.PRIM_SPHERE, Q // 4, Q // 4, Q // 4, Q // 10, 0, 0, 0]], np.int64)
    t = oracle.build_tree(prims, 1)
    assert t["child"].shape == (1, 8)
    assert list(t["child"][0]) == [-1, -2, -3, -4, -5, -6, -7, -8]
    assert list(t["leaf_key"]) == list(range(8, 16))
    assert list(t["leaf_inside"]) == [1, 0, 0, 0, 0, 0, 0, 0]
    assert list(t["node_parent"]) == [-1]
    assert list(t["leaf_parent"]) == [0] * 8


def test_depth2_box_by_hand():
    # box (0.3..0.45)^3 lies inside octant 0, and inside its level-2 child (1,1,1) only
    lo, hi = int(0.3 * Q), int(0.45 * Q)
    prims = np.array([[si.PRIM_BOX, lo, lo, lo, hi, hi, hi, 0]], np.int64)
    t = oracle.build_tree(prims, 2)
    assert t["child"].shape[0] == 2
    assert t["child"][0, 0] == 1            # octant 0 is internal node 1
    assert list(t["child"][0, 1:]) == [-1, -2, -3, -4, -5, -6, -7]
    # node 1's children are leaves 7..14; slot 7 = (1,1,1) is the only inside leaf
    assert list(t["child"][1]) == [-8, -9, -10, -11, -12, -13, -14, -15]
    assert t["leaf_inside"].tolist() == [0] * 7 + [0] * 7 + [1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_structure_matches_bruteforce(seed):
    sc = si.random_scene(seed, max_depth=4, n_prims=4)
    t = oracle.scene_tree(sc)
    D = sc.max_depth
    internal = {int(k) for k in t["node_key"]}
    leaves = {int(k) for k in t["leaf_key"]}
    assert len(internal) == t["node_key"].size and len(leaves) == t["leaf_key"].size
    # brute force per level: a cell exists iff its parent is internal; it is internal iff it
    # meets the scene and is above D (the root always)
    expect_internal, expect_leaf, expect_inside = {1}, set(), set()
    frontier = [1]
    for l in range(1, D + 1):
        cells = [(p << 3) | j for p in frontier for j in range(8)]
        ks = np.array([_decode(c)[1] for c in cells], np.int64)
        m = _meets_bruteforce(sc.prims, l, ks[:, 0], ks[:, 1], ks[:, 2])
        frontier = []
        for c, mi in zip(cells, m):
            if mi and l < D:
                expect_internal.add(c)
                frontier.append(c)
            else:
                expect_leaf.add(c)
                if mi:
                    expect_inside.add(c)
    assert internal == expect_internal
    assert leaves == expect_leaf
    inside = {int(k) for k, f in zip(t["leaf_key"], t["leaf_inside"]) if f}
    assert inside == expect_inside


@pytest.mark.parametrize("seed", [4, 5])
def test_volume_partition_and_point_location(seed):
    sc = si.random_scene(seed, max_depth=5, n_prims=3)
    t = oracle.scene_tree(sc)
    # leaf volumes (in finest cells) sum exactly to the root volume
    lv = oracle.key_level(t["leaf_key"])
    D = int(lv.max())
    assert int(np.sum(8 ** (D - lv))) == 8 ** D
    # every point lies in exactly one leaf: descend by child pointers, then check the cell
    rng = np.random.default_rng(seed)
    P = rng.random((2000, 3))
    key_of = t["leaf_key"]
    for p in P:
        node, l, k = 0, 0, np.zeros(3, np.int64)
        while True:
            b = (p * (1 << (l + 1))).astype(np.int64) & 1
            j = 4 * b[0] + 2 * b[1] + b[2]
            ch = t["child"][node, j]
            k = 2 * k + b
            l += 1
            if ch < 0:
                v = -1 - ch
                lv_, kv = _decode(key_of[v])
                assert lv_ == l and list(kv) == list(k)
                assert np.all(p >= np.array(kv) / (1 << l)) and np.all(p < (np.array(kv) + 1) / (1 << l))
                break
            node = ch


def test_canonical_bfs_morton_order():
    sc = si.random_scene(9, max_depth=5, n_prims=4)
    t = oracle.scene_tree(sc)
    for name in ("node_key", "leaf_key"):
        keys = t[name].astype(np.uint64)
        lv = oracle.key_level(keys)
        assert np.all(np.diff(lv) >= 0)
        same = lv[1:] == lv[:-1]
        assert np.all(keys[1:][same] > keys[:-1][same])
    # child pointers agree with keys and parents
    for p in range(t["child"].shape[0]):
        for j in range(8):
            ch = t["child"][p, j]
            if ch >= 0:
                assert t["node_key"][ch] == (int(t["node_key"][p]) << 3) | j
                assert t["node_parent"][ch] == p
            else:
                assert t["leaf_key"][-1 - ch] == (int(t["node_key"][p]) << 3) | j
                assert t["leaf_parent"][-1 - ch] == p


def test_config_scene_sizes():
    sc, _ = si.config_tiny()
    t = oracle.scene_tree(sc)
    assert 100 <= t["leaf_key"].size <= 2000
