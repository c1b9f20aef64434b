"""Pins of the oracle's median-cut quantiser of SH coefficient vectors (Heckbert 1982, applied in
Sec. 4.1 to build the compressed models), no GPU: hand-worked splits, the longest-axis and tie
rules, clustered data reconstructed exactly, nested refinement lowering the squared error, and the
rendering of a compressed tree equal to the rendering of its expanded coefficients."""
import numpy as np

import oracle
import seeded_inputs as si


def test_one_dimension_by_hand():
    x = np.array([[0.0], [1.0], [2.0], [3.0], [10.0], [11.0], [12.0], [13.0]])
    idx, pal = oracle.median_cut(x, 2)
    assert idx.tolist() == [0, 0, 1, 1, 2, 2, 3, 3]
    np.testing.assert_array_equal(pal[:, 0], [0.5, 2.5, 10.5, 12.5])
    idx, pal = oracle.median_cut(x[::-1].copy(), 1)
    assert idx.tolist() == [1, 1, 1, 1, 0, 0, 0, 0]
    np.testing.assert_array_equal(pal[:, 0], [1.5, 11.5])


def test_split_follows_the_longest_axis():
    """Axis 1 spans 30 and axis 0 only 3: the halves are the two smallest and two largest y."""
    x = np.array([[0.0, 30.0], [1.0, 0.0], [2.0, 20.0], [3.0, 10.0]])
    idx, pal = oracle.median_cut(x, 1)
    assert idx.tolist() == [1, 0, 1, 0]
    np.testing.assert_array_equal(pal, [[2.0, 5.0], [1.0, 25.0]])


def test_ties_and_odd_counts():
    idx, pal = oracle.median_cut(np.ones((4, 3)), 1)
    assert idx.tolist() == [0, 0, 1, 1]          # equal values: vector id decides
    idx, _ = oracle.median_cut(np.arange(5.0)[:, None], 1)
    assert idx.tolist() == [0, 0, 1, 1, 1]       # floor(5 / 2) to the lower child
    idx, pal = oracle.median_cut(np.array([[2.0]]), 3)
    assert idx.tolist() == [0] and pal[0, 0] == 2.0 and not pal[1:].any()


def test_clusters_are_reconstructed_exactly():
    rng = np.random.default_rng(0)
    P, k, dim = 16, 7, 12
    centers = rng.normal(size=(P, dim)) * 10
    x = np.repeat(centers, k, axis=0)
    perm = rng.permutation(P * k)
    x = x[perm]
    idx, pal = oracle.median_cut(x, 4)
    np.testing.assert_allclose(pal[idx], x, atol=1e-12)
    assert np.unique(idx).size == P


def test_box_sizes_and_palette_means():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(64 * 5, 9))
    idx, pal = oracle.median_cut(x, 6)
    assert (np.bincount(idx, minlength=64) == 5).all()
    for b in range(64):
        np.testing.assert_allclose(pal[b], x[idx == b].mean(axis=0), rtol=1e-13, atol=1e-15)


def test_refinement_lowers_the_squared_error():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1000, 6)) * rng.random(6)
    sse = []
    for bits in range(0, 11):
        idx, pal = oracle.median_cut(x, bits)
        sse.append(((pal[idx] - x) ** 2).sum())
        if bits:
            prev = oracle.median_cut(x, bits - 1)[0]
            assert np.array_equal(idx >> 1, prev)     # boxes nest: each splits its parent
    assert all(b <= a + 1e-9 for a, b in zip(sse, sse[1:]))
    assert sse[-1] < 0.2 * sse[0]


def test_compressed_render_equals_expanded_render():
    """A compressed tree renders with sh[v] = palette[index[v]]: the oracle's render of the
    expanded coefficients is the definition; quantising to 2^bits >= L boxes loses nothing."""
    sc = si.random_scene(5, max_depth=3, sh_degree=2, n_prims=2)
    t = oracle.scene_tree(sc)
    sig, sh = si.leaf_params(t["leaf_key"], t["leaf_inside"], sc)
    s64, h64 = si.storage_to_f64(sig, sc.storage), si.storage_to_f64(sh, sc.storage)
    L = s64.size
    bits = int(np.ceil(np.log2(L)))
    idx, pal = oracle.median_cut(h64.reshape(L, -1), bits)
    np.testing.assert_allclose(pal[idx].reshape(h64.shape), h64, atol=1e-15)
    lo, size = oracle.root_of(sc)
    o, d = si.random_rays(200, 3)
    a, _, _ = oracle.render(t, lo, size, s64, h64, 2, o, d)
    b, _, _ = oracle.render(t, lo, size, s64, pal[idx].reshape(h64.shape), 2, o, d)
    np.testing.assert_allclose(a, b, atol=1e-14)
