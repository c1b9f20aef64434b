"""Pins of the oracle's selection (Sec. 3.2, Algorithm 1) and prune / sample (Eq. 3-4), no GPU.

Hand-built trees with outputs written out by hand, library sorts for the top-k, and rendering
invariants: subdivision by copy and the prune of identical children leave every pixel unchanged,
and sampling everything then pruning everything gives back the original tree.
"""
import numpy as np
import pytest

import oracle
import seeded_inputs as si

Q = si.Q


def _depth1_tree():
    prims = np.array([[si.PRIM_SPHERE, Q // 4, Q // 4, Q // 4, Q // 10, 0, 0, 0]], np.int64)
    return oracle.build_tree(prims, 1)


def test_sample_one_leaf_by_hand():
    t = _depth1_tree()
    sigma = np.arange(8, dtype=np.float64) + 1
    sh = np.arange(8 * 3, dtype=np.float64).reshape(8, 3, 1)
    prune = np.zeros(8, np.uint8)
    sample = np.zeros(8, np.uint8)
    sample[3] = 1
    new, lm, so, sho, cnt = oracle.refine(t, sigma, sh, prune, sample, d_cap=8)
    assert cnt == {"n_nodes": 2, "n_leaves": 15, "n_pruned_groups": 0, "n_sampled": 1, "n_capped": 0}
    assert new["child"].tolist() == [[-1, -2, -3, 1, -4, -5, -6, -7],
                                     [-8, -9, -10, -11, -12, -13, -14, -15]]
    assert new["node_parent"].tolist() == [-1, 0]
    assert new["node_key"].tolist() == [1, 11]
    assert lm.tolist() == [0, 1, 2, 4, 5, 6, 7] + [3] * 8
    assert new["leaf_key"].tolist() == [8, 9, 10, 12, 13, 14, 15] + [(11 << 3) | j for j in range(8)]
    assert new["leaf_parent"].tolist() == [0] * 7 + [1] * 8
    np.testing.assert_array_equal(so, sigma[lm])
    np.testing.assert_array_equal(sho, sh[lm])

    # prune the 8 new children back: the merged parent becomes leaf 7 (after the 7 survivors)
    p2 = np.zeros(15, np.uint8)
    p2[7:] = 1
    s2 = np.zeros(15, np.uint8)
    new2, lm2, so2, sho2, cnt2 = oracle.refine(new, so, sho, p2, s2, d_cap=8)
    assert cnt2["n_pruned_groups"] == 1 and cnt2["n_nodes"] == 1 and cnt2["n_leaves"] == 8
    assert new2["child"].tolist() == [[-1, -2, -3, -8, -4, -5, -6, -7]]
    assert lm2.tolist() == [0, 1, 2, 3, 4, 5, 6, -2]          # -1 - (old node 1)
    assert new2["leaf_key"].tolist() == [8, 9, 10, 12, 13, 14, 15, 11]
    assert so2[7] == sigma[3] and np.array_equal(sho2[7], sh[3])


def test_root_never_merged_and_depth_cap():
    t = _depth1_tree()
    sigma = np.ones(8)
    sh = np.ones((8, 3, 1))
    new, lm, _, _, cnt = oracle.refine(t, sigma, sh, np.ones(8, np.uint8), np.zeros(8, np.uint8), 8)
    assert cnt["n_pruned_groups"] == 0 and new["child"].tolist() == t["child"].tolist()
    assert lm.tolist() == list(range(8))
    s = np.zeros(8, np.uint8)
    s[[1, 5]] = 1
    new, lm, _, _, cnt = oracle.refine(t, sigma, sh, np.zeros(8, np.uint8), s, d_cap=1)
    assert cnt["n_capped"] == 2 and cnt["n_sampled"] == 0 and cnt["n_leaves"] == 8


def test_prune_rules_depth2():
    """Depth-2 tree with 2 internal children of the root: merge only where all 8 children are
    prune-marked and none is sample-marked."""
    lo1, hi1 = int(0.05 * Q), int(0.2 * Q)
    lo2, hi2 = int(0.8 * Q), int(0.95 * Q)
    prims = np.array([[si.PRIM_BOX, lo1, lo1, lo1, hi1, hi1, hi1, 0],
                      [si.PRIM_BOX, lo2, lo2, lo2, hi2, hi2, hi2, 0]], np.int64)
    t = oracle.build_tree(prims, 2)
    assert t["child"].shape[0] == 3                 # root, octant 0, octant 7
    L = t["leaf_key"].size                          # 6 level-1 leaves + 16 level-2 leaves
    assert L == 22
    sigma = np.arange(L, dtype=np.float64)
    sh = np.zeros((L, 3, 1))
    prune = np.ones(L, np.uint8)
    sample = np.zeros(L, np.uint8)
    sample[6 + 8 + 2] = 1                           # a child of node 2 (octant 7) sample-marked
    new, lm, so, _, cnt = oracle.refine(t, sigma, sh, prune, sample, d_cap=5)
    # node 1 merged (leaf ids 6..13), node 2 kept and its slot-2 child sampled
    assert cnt["n_pruned_groups"] == 1 and cnt["n_sampled"] == 1
    assert cnt["n_nodes"] == 3 and cnt["n_leaves"] == 6 + 7 + 1 + 8
    assert lm.tolist() == [0, 1, 2, 3, 4, 5] + [14, 15, 17, 18, 19, 20, 21] + [-2] + [16] * 8
    assert so[13] == pytest.approx(np.mean(sigma[6:14]))
    # root: slot 0 -> merged leaf (new id 13), slots 1..6 -> leaves 0..5, slot 7 -> node 1
    assert new["child"][0].tolist() == [-14, -1, -2, -3, -4, -5, -6, 1]
    assert new["child"][1].tolist() == [-7, -8, 2, -9, -10, -11, -12, -13]
    assert new["child"][2].tolist() == [-15 - j for j in range(8)]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sample_by_copy_leaves_pixels_unchanged(seed):
    sc = si.random_scene(seed, max_depth=3, sh_degree=2, n_prims=3)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(0, 5, L)
    sh = rng.normal(0, 0.5, (L, 3, 9))
    o, d = si.random_rays(200, seed + 3)
    rgb0, T0, _ = oracle.render(t, lo, size, sigma, sh, 2, o, d, eps_T=0.0)
    sample = (rng.random(L) < 0.5).astype(np.uint8)
    new, lm, so, sho, cnt = oracle.refine(t, sigma, sh, np.zeros(L, np.uint8), sample, 8)
    rgb1, T1, _ = oracle.render(new, lo, size, so, sho, 2, o, d, eps_T=0.0)
    np.testing.assert_allclose(rgb1, rgb0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(T1, T0, rtol=1e-12, atol=1e-15)
    # gradient additivity: the children's gradients sum to the parent's
    g = rng.normal(size=(200, 3))
    gs0, gsh0, _, _ = oracle.backward(t, lo, size, sigma, sh, 2, o, d, g, eps_T=0.0)
    gs1, gsh1, _, _ = oracle.backward(new, lo, size, so, sho, 2, o, d, g, eps_T=0.0)
    back_s = np.zeros(L)
    back_sh = np.zeros_like(sh)
    np.add.at(back_s, lm, gs1)
    np.add.at(back_sh, lm, gsh1)
    np.testing.assert_allclose(back_s, gs0, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(back_sh, gsh0, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("seed", [3, 4])
def test_sample_all_then_prune_all_is_identity(seed):
    sc = si.random_scene(seed, max_depth=3, sh_degree=1, n_prims=2)
    t = oracle.scene_tree(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(seed)
    sigma = rng.uniform(0, 5, L)
    sh = rng.normal(0, 0.5, (L, 3, 4))
    new, lm, so, sho, _ = oracle.refine(t, sigma, sh, np.zeros(L, np.uint8), np.ones(L, np.uint8), 8)
    L2 = new["leaf_key"].size
    assert L2 == 8 * L
    back, lm2, so2, sho2, cnt = oracle.refine(new, so, sho, np.ones(L2, np.uint8),
                                              np.zeros(L2, np.uint8), 8)
    for k in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        np.testing.assert_array_equal(back[k], t[k])
    np.testing.assert_array_equal(so2, sigma)       # mean of 8 identical values is exact
    np.testing.assert_array_equal(sho2, sh)


def test_prune_identical_children_leaves_pixels_unchanged():
    sc = si.random_scene(8, max_depth=4, sh_degree=1, n_prims=3)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(8)
    sigma = rng.uniform(0, 5, L)
    sh = rng.normal(0, 0.5, (L, 3, 4))
    # make every all-leaf sibling group identical, then prune them all
    prune = np.zeros(L, np.uint8)
    for p in range(1, t["child"].shape[0]):
        ch = t["child"][p]
        if np.all(ch < 0):
            v = -1 - ch
            sigma[v] = sigma[v[0]]
            sh[v] = sh[v[0]]
            prune[v] = 1
    o, d = si.random_rays(200, 5)
    rgb0, _, _ = oracle.render(t, lo, size, sigma, sh, 1, o, d, eps_T=0.0)
    new, lm, so, sho, cnt = oracle.refine(t, sigma, sh, prune, np.zeros(L, np.uint8), 8)
    assert cnt["n_pruned_groups"] > 0
    rgb1, _, _ = oracle.render(new, lo, size, so, sho, 1, o, d, eps_T=0.0)
    np.testing.assert_allclose(rgb1, rgb0, rtol=0, atol=1e-12)


def test_select_threshold_and_rank():
    s = si.random_signal(5000, 1)
    pm, sm = oracle.select(s, oracle.SELECT_THRESHOLD, 0.3, oracle.SELECT_THRESHOLD, 2.0)
    np.testing.assert_array_equal(pm, (s <= np.float32(0.3)).astype(np.uint8))
    np.testing.assert_array_equal(sm, (s > np.float32(2.0)).astype(np.uint8))
    for frac in (0.0, 0.01, 0.05, 0.2, 1.0):
        pm, sm = oracle.select(s, oracle.SELECT_FRACTION, frac, oracle.SELECT_FRACTION, frac)
        k = int(np.ceil(frac * s.size))
        ids = np.arange(s.size)
        top = np.lexsort((ids, -s.astype(np.float64)))[:k]       # S desc, id asc
        bot = np.lexsort((ids, s.astype(np.float64)))[:k]        # S asc, id asc
        e = np.zeros(s.size, np.uint8)
        e[top] = 1
        np.testing.assert_array_equal(sm, e)
        e = np.zeros(s.size, np.uint8)
        e[bot] = 1
        np.testing.assert_array_equal(pm, e)


def _brute_rank_marks(s, frac, desc, ties=False):
    """Marks of the ceil(frac n) first leaves in the selection order, by a plain Python sort:
    NaN after every number, -0.0 == +0.0 (Python float equality), then leaf id.  With ties, also
    every leaf whose (NaN flag, value) equals the k-th one's."""
    n = len(s)
    k = int(np.ceil(frac * n))

    def key(i):
        x = float(s[i])
        if x != x:
            return (1, 0.0, i)
        return (0, -x if desc else x, i)
    order = sorted(range(n), key=key)
    m = np.zeros(n, np.uint8)
    m[order[:k]] = 1
    if ties and k > 0:
        last = key(order[k - 1])[:2]
        for i in range(n):
            if key(i)[:2] == last:
                m[i] = 1
    return m


def test_select_signed_zeros_and_nan():
    """Signed zeros are one value and a NaN sorts last in both directions; a k-th boundary that
    falls inside a run of mixed +0.0 / -0.0 signals is filled in leaf-id order."""
    rng = np.random.default_rng(3)
    n = 400
    s = rng.exponential(1.0, n).astype(np.float32)
    zeros = rng.choice(n, 120, replace=False)
    s[zeros] = np.where(rng.random(120) < 0.5, np.float32(-0.0), np.float32(0.0))
    rest = np.setdiff1d(np.arange(n), zeros)
    s[rng.choice(rest, 9, replace=False)] = np.nan
    assert np.any(np.signbit(s) & (s == 0)) and np.any(~np.signbit(s) & (s == 0))
    for frac in (0.1, 0.2, 0.3, 0.5, 0.98, 1.0):
        pm, sm = oracle.select(s, oracle.SELECT_FRACTION, frac, oracle.SELECT_FRACTION, frac)
        np.testing.assert_array_equal(pm, _brute_rank_marks(s, frac, False))
        np.testing.assert_array_equal(sm, _brute_rank_marks(s, frac, True))
        pm, sm = oracle.select(s, oracle.SELECT_QUANTILE, frac, oracle.SELECT_QUANTILE, frac)
        np.testing.assert_array_equal(pm, _brute_rank_marks(s, frac, False, ties=True))
        np.testing.assert_array_equal(sm, _brute_rank_marks(s, frac, True, ties=True))
    # the bottom 10% / 20% boundary lies inside the 120 zeros: both signs are taken by id
    pm, _ = oracle.select(s, oracle.SELECT_FRACTION, 0.2, oracle.SELECT_NONE, 0.0)
    zsorted = np.sort(zeros)
    np.testing.assert_array_equal(np.flatnonzero(pm), zsorted[:80])
    # a NaN is never marked by a threshold, and is picked last by a rank selection
    pm, sm = oracle.select(s, oracle.SELECT_THRESHOLD, np.inf, oracle.SELECT_THRESHOLD, -np.inf)
    assert not np.any(pm[np.isnan(s)]) and not np.any(sm[np.isnan(s)])
    _, sm = oracle.select(s, oracle.SELECT_NONE, 0.0, oracle.SELECT_FRACTION, (n - 9) / n)
    assert not np.any(sm[np.isnan(s)]) and sm.sum() == n - 9
    # the quantile of a boundary inside the zeros takes every zero of either sign, and the
    # quantile prune equals a threshold at the k-th value
    pm, _ = oracle.select(s, oracle.SELECT_QUANTILE, 0.2, oracle.SELECT_NONE, 0.0)
    np.testing.assert_array_equal(np.flatnonzero(pm), np.sort(zeros))
    for frac in (0.05, 0.4, 0.7):
        k = int(np.ceil(frac * n))
        kth = np.sort(s[~np.isnan(s)])[k - 1]
        pm, _ = oracle.select(s, oracle.SELECT_QUANTILE, frac, oracle.SELECT_NONE, 0.0)
        np.testing.assert_array_equal(pm, (s <= kth).astype(np.uint8))


# ----------------------------------------------------------------------------------------------
# recursive pruning (Sec. 3.2, Algorithm 1 with rec)
# ----------------------------------------------------------------------------------------------
def _full_depth3():
    """Every cell of a depth-3 tree meets the box [0, 1]^3 -> 1 + 8 + 64 nodes, 512 leaves."""
    prims = np.array([[si.PRIM_BOX, 0, 0, 0, Q, Q, Q, 0]], np.int64)
    t = oracle.build_tree(prims, 3)
    assert t["leaf_key"].size == 512 and t["node_key"].size == 73
    return t


def test_recursive_prune_of_a_silent_tree_collapses_to_the_root():
    t = _full_depth3()
    rng = np.random.default_rng(0)
    sigma = rng.uniform(1, 2, 512)
    sh = rng.normal(size=(512, 3, 1))
    sig = np.zeros(512, np.float32)
    nt, so, sho, s2, _, passes = oracle.prune_recursive(t, sigma, sh, sig, 0.0, d_cap=8)
    assert [p["n_pruned_groups"] for p in passes] == [64, 8]
    assert nt["leaf_key"].size == 8 and nt["node_key"].size == 1
    # each level-1 leaf holds the mean of the 64 finest leaves below it (Eq. 3 applied twice)
    keys = t["leaf_key"]
    for u, k in enumerate(nt["leaf_key"]):
        below = (keys >> np.uint64(6)) == k
        assert below.sum() == 64
        assert so[u] == pytest.approx(sigma[below].mean(), rel=1e-14)
        np.testing.assert_allclose(sho[u], sh[below].mean(axis=0), rtol=1e-13, atol=1e-15)
    one = oracle.prune_recursive(t, sigma, sh, sig, 0.0, d_cap=8, recursive=False)
    assert [p["n_pruned_groups"] for p in one[5]] == [64] and one[0]["leaf_key"].size == 64


@pytest.mark.parametrize("merge,expect_passes,n_leaves",
                         [("sum", [511, 63], 63 + 7 + 8), ("max", [511, 63, 7], 7 + 7 + 7 + 8)])
def test_recursive_prune_merged_signal(merge, expect_passes, n_leaves):
    """Full depth-4 tree; one loud leaf (1.0) blocks its group, quiet leaves carry 0.01, tau = 0.5.
    Each pass thresholds the current leaves: merged parents carry 0.08 then 0.64 with sum (the
    third pass finds 0.64 > tau and stops) or stay at 0.01 with max (the third pass merges the 7
    level-1 cells whose children are all leaves)."""
    prims = np.array([[si.PRIM_BOX, 0, 0, 0, Q, Q, Q, 0]], np.int64)
    t = oracle.build_tree(prims, 4)
    assert t["leaf_key"].size == 4096
    sigma = np.ones(4096)
    sh = np.zeros((4096, 3, 1))
    sig = np.full(4096, 0.01, np.float32)
    sig[1234] = 1.0
    nt, _, _, s2, _, passes = oracle.prune_recursive(t, sigma, sh, sig, 0.5, d_cap=8, merge=merge)
    assert [p["n_pruned_groups"] for p in passes] == expect_passes
    assert nt["leaf_key"].size == n_leaves
    assert s2.max() == pytest.approx(1.0)
    assert np.isin(t["leaf_key"][1234], nt["leaf_key"])
    if merge == "sum":
        assert np.sort(s2)[-2] == pytest.approx(0.64, rel=1e-6)


def test_remap_leaf_values_by_hand():
    t = _depth1_tree()
    nt, lm, _, _, _ = oracle.refine(t, np.ones(8), np.zeros((8, 3, 1)), np.ones(8, np.uint8),
                                    np.zeros(8, np.uint8), d_cap=8)
    # the root is never merged: nothing changes
    assert lm.tolist() == list(range(8))
    s = np.arange(8, dtype=np.float64)
    np.testing.assert_array_equal(oracle.remap_leaf_values(t, lm, s), s)


# ----------------------------------------------------------------------------------------------
# canonical numbering after refines
# ----------------------------------------------------------------------------------------------
def _consistent(t):
    """Every pointer agrees with the keys: child slot j of key k holds key (k << 3) | j."""
    child, nk, lk = t["child"], t["node_key"], t["leaf_key"]
    for n in range(nk.size):
        for j in range(8):
            c = int(child[n, j])
            key = int(nk[c]) if c >= 0 else int(lk[-1 - c])
            assert key == (int(nk[n]) << 3) | j
            par = t["node_parent"][c] if c >= 0 else t["leaf_parent"][-1 - c]
            assert par == n


def test_canonical_form_of_a_built_tree_is_itself():
    sc = si.random_scene(3, max_depth=4, sh_degree=0, n_prims=3)
    t = oracle.scene_tree(sc)
    new, perm, _ = oracle.canonicalize(t)
    assert perm.tolist() == list(range(t["leaf_key"].size))
    for k in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        assert np.array_equal(new[k], t[k]), k


def test_canonical_form_after_refines_is_sorted_and_consistent():
    sc = si.random_scene(4, max_depth=4, sh_degree=1, n_prims=3)
    t = oracle.scene_tree(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(0)
    sigma = rng.random(L)
    sh = rng.normal(size=(L, 3, 4))
    for r in range(3):
        L = t["leaf_key"].size
        pm = (rng.random(L) < 0.5).astype(np.uint8)
        sm = (rng.random(L) < 0.1).astype(np.uint8)
        t, lm, sigma, sh, _ = oracle.refine(t, sigma, sh, pm, sm, 7)
    assert np.any(np.diff(t["leaf_key"].astype(np.int64)) < 0)       # refines append
    new, perm, (s2, h2) = oracle.canonicalize(t, (sigma, sh))
    assert np.all(np.diff(new["leaf_key"].astype(np.int64)) > 0)
    assert np.all(np.diff(new["node_key"].astype(np.int64)) > 0)
    assert new["node_key"][0] == 1 and new["node_parent"][0] == -1
    _consistent(new)
    np.testing.assert_array_equal(s2, sigma[perm])
    # the same cells render the same: rays see identical segments and values
    lo, size = oracle.root_of(sc)
    o, d = si.random_rays(100, 5)
    a, _, _ = oracle.render(t, lo, size, sigma, sh, 1, o, d)
    b, _, _ = oracle.render(new, lo, size, s2, h2, 1, o, d)
    np.testing.assert_array_equal(a, b)
