"""The face-neighbour table of a tree (ropes), bit-exact against an independent computation from
the exported keys, after build, refine, canonical renumbering and import."""
import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu

INT32_MIN = -(1 << 31)


def _level_coords(key):
    key = int(key)
    lv = (key.bit_length() - 1) // 3
    k = key & ((1 << 3 * lv) - 1)
    c = [0, 0, 0]
    for b in range(lv):
        tri = (k >> (3 * (lv - 1 - b))) & 7
        c = [(c[0] << 1) | (tri >> 2), (c[1] << 1) | ((tri >> 1) & 1), (c[2] << 1) | (tri & 1)]
    return lv, c


def _key(lv, c):
    k = 1
    for b in range(lv - 1, -1, -1):
        k = (k << 3) | (((c[0] >> b) & 1) << 2) | (((c[1] >> b) & 1) << 1) | ((c[2] >> b) & 1)
    return k


def expected_ropes(ex, leaves):
    """For each leaf of `leaves` and each face: the cell across the face at the leaf's level,
    looked up by key -- a node with that key, else the leaf whose key is an ancestor key of it
    (a coarser cell)."""
    node_of = {int(k): i for i, k in enumerate(ex["node_key"])}
    leaf_of = {int(k): i for i, k in enumerate(ex["leaf_key"])}
    out = np.empty((len(leaves), 6), np.int64)
    for row, v in enumerate(leaves):
        lv, c = _level_coords(ex["leaf_key"][v])
        for f in range(6):
            a = f >> 1
            n = list(c)
            n[a] += 1 if f & 1 else -1
            if not 0 <= n[a] < (1 << lv):
                out[row, f] = INT32_MIN
                continue
            k = _key(lv, n)
            if k in node_of:
                out[row, f] = node_of[k]
                continue
            for m in range(lv, 0, -1):
                km = _key(m, [x >> (lv - m) for x in n])
                if km in leaf_of:
                    out[row, f] = -1 - ((leaf_of[km] << 4) | (lv - m))
                    break
            else:
                raise AssertionError("no cell covers the neighbour")
    return out


def _check(tree, sample=None):
    torch.cuda.synchronize()
    got = tree.rope.cpu().numpy().astype(np.int64)
    L = got.shape[0]
    leaves = np.arange(L) if sample is None else np.random.default_rng(9).choice(L, sample, False)
    np.testing.assert_array_equal(got[leaves], expected_ropes(tree.export(), leaves))
    return got


def test_ropes_after_build_refine_canonicalize_import():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(31, max_depth=6, sh_degree=1, storage=si.STORAGE_F16, n_prims=4)
    tree = dot.octree_from_scene(scene)
    got = _check(tree)
    assert (got >= 0).any() and (got == INT32_MIN).any() and ((got < 0) & (got != INT32_MIN)).any()
    assert (((-1 - got[(got < 0) & (got != INT32_MIN)]) & 15) > 0).any()  # coarser neighbours
    rng = np.random.default_rng(5)
    for r in range(2):
        L = tree.n_leaves
        pm = torch.from_numpy((rng.random(L) < 0.6).astype(np.uint8)).cuda()
        sm = torch.from_numpy((rng.random(L) < 0.05).astype(np.uint8)).cuda()
        plan = dot.dot_refine_plan(tree, pm, sm, 8)
        dot.dot_refine_prune(tree, pm, sm, 8, torch.empty(plan["n_leaves"], dtype=torch.int32,
                                                            device="cuda"))
        _check(tree)
    dot.dot.dot_tree_canonicalize(tree, torch.empty(tree.n_leaves, dtype=torch.int32, device="cuda"))
    _check(tree)
    imported = dot.dot_tree_import(tree.export())
    np.testing.assert_array_equal(_check(imported), tree.rope.cpu().numpy())
    imported.free()
    tree.free()


def test_ropes_of_a_deep_tree():
    import paper_2307_15333_gb300 as dot
    c = (0.1, -0.05, 0.02)
    prims = si._prims([si.sphere(c, 0.0006, (0.0, 0.0, 0.0), 1.0)])
    scene = si.Scene("deep16", (0.0, 0.0, 0.0), 1.0, 16, 0, si.STORAGE_F32, prims, 5.0, 50.0, 0.4,
                     0.2, 3)
    tree = dot.octree_from_scene(scene)
    got = _check(tree)
    d = (-1 - got[(got < 0) & (got != INT32_MIN)]) & 15
    assert d.max() >= 5                                   # neighbours several levels coarser
    tree.free()
