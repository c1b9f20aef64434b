"""GPU selection (Sec. 3.2 / Algorithm 1) and prune / sample (Eq. 3-4) vs the oracle: masks,
structure and leaf maps bit-exact, merged means within one unit in the last place of storage."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import bits, oracle_side

pytestmark = pytest.mark.gpu


def _tree(scene):
    import paper_2307_15333_gb300 as dot
    return dot.octree_from_scene(scene)


@pytest.mark.parametrize("D", [1, 2, 4, 6, 7])
def test_select_sizes(D):
    import paper_2307_15333_gb300 as dot
    scene = si.box_scene((-2, -2, -2), (2, 2, 2), max_depth=D, sh_degree=0)
    tree = _tree(scene)
    L = tree.n_leaves
    s = si.random_signal(L, D)
    sig = torch.from_numpy(s).cuda()
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    for (pmode, pval, smode, sval) in [(2, 0.0, 2, 0.01), (2, 0.2, 2, 0.05), (2, 1.0, 2, 1.0),
                                       (1, 0.3, 1, 2.0), (2, 0.5, 0, 0.0), (0, 0.0, 2, 0.999),
                                       (3, 0.2, 3, 0.05), (3, 0.0, 3, 1.0), (3, 0.9, 2, 0.3)]:
        dot.dot_select_masks(tree, sig, dot.select_opts(pmode, pval, smode, sval), pm, sm)
        rp, rs = oracle.select(s, pmode, pval, smode, sval)
        np.testing.assert_array_equal(pm.cpu().numpy(), rp)
        np.testing.assert_array_equal(sm.cpu().numpy(), rs)
    tree.free()


def _compare_refine(scene, prune, sample, d_cap, aux_width=0):
    import paper_2307_15333_gb300 as dot
    tree = _tree(scene)
    t, sig, sh, s64, h64 = oracle_side(scene)
    L = t["leaf_key"].size
    K = scene.n_coeffs
    pm = torch.from_numpy(prune).cuda()
    sm = torch.from_numpy(sample).cuda()
    counts = dot.dot_refine_plan(tree, pm, sm, d_cap)
    new, lm, so, sho, oc = oracle.refine(t, s64, h64.reshape(L, -1), prune, sample, d_cap)
    assert counts == {"n_nodes": oc["n_nodes"], "n_leaves": oc["n_leaves"],
                      "n_pruned_groups": oc["n_pruned_groups"], "n_sampled": oc["n_sampled"],
                      "n_capped": oc["n_capped"]}
    leaf_map = torch.empty(counts["n_leaves"], dtype=torch.int32, device="cuda")
    aux = []
    if aux_width:
        src = torch.randn(L, aux_width, device="cuda")
        dst_mean = torch.empty(counts["n_leaves"], aux_width, device="cuda")
        dst_max = torch.empty(counts["n_leaves"], aux_width, device="cuda")
        aux = [(src, dst_mean, dot.dot.DOT_MERGE_MEAN), (src, dst_max, dot.dot.DOT_MERGE_MAX)]
    dot.dot_refine_prune(tree, pm, sm, d_cap, leaf_map, aux)
    ex = tree.export()
    for k in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        np.testing.assert_array_equal(ex[k], new[k], err_msg=k)
    np.testing.assert_array_equal(leaf_map.cpu().numpy(), lm)
    # copies are exact; merged means within one unit of the storage's last place
    copy = lm >= 0
    np.testing.assert_array_equal(bits(ex["sigma"][copy]), bits(sig[lm[copy]]))
    np.testing.assert_array_equal(bits(ex["sh"][copy]), bits(sh[lm[copy]]))
    got_s = si.storage_to_f64(ex["sigma"], scene.storage)
    got_h = si.storage_to_f64(ex["sh"], scene.storage).reshape(len(lm), -1)
    ulp = {si.STORAGE_F32: 2.0 ** -23, si.STORAGE_F16: 2.0 ** -10, si.STORAGE_BF16: 2.0 ** -7}[scene.storage]
    ref_h = sho.reshape(len(lm), -1)
    h64f = h64.reshape(L, -1)
    for u in np.nonzero(lm < 0)[0]:
        kids = -1 - t["child"][-1 - lm[u]]
        # pairwise FP32 sum of 8 values, then one rounding to storage
        lim_s = 4 * ulp * np.abs(s64[kids]).max() + 2.0 ** -24
        lim_h = 4 * ulp * np.abs(h64f[kids]).max(0) + 2.0 ** -24
        assert abs(got_s[u] - so[u]) <= lim_s
        assert np.all(np.abs(got_h[u] - ref_h[u]) <= lim_h)
    if aux_width:
        s_np = aux[0][0].cpu().numpy().astype(np.float64)
        mean_ref = np.empty((len(lm), aux_width))
        max_ref = np.empty((len(lm), aux_width))
        for u, src_id in enumerate(lm):
            if src_id >= 0:
                mean_ref[u] = max_ref[u] = s_np[src_id]
            else:
                kids = -1 - t["child"][-1 - src_id]
                mean_ref[u] = s_np[kids].mean(0)
                max_ref[u] = s_np[kids].max(0)
        np.testing.assert_allclose(aux[0][1].cpu().numpy(), mean_ref, rtol=1e-6, atol=1e-6)
        np.testing.assert_array_equal(aux[1][1].cpu().numpy(), max_ref.astype(np.float32))
    assert ex["max_level"] == int(oracle.key_level(new["leaf_key"]).max())
    tree.free()
    return counts


@pytest.mark.parametrize("storage", [si.STORAGE_F32, si.STORAGE_F16, si.STORAGE_BF16])
@pytest.mark.parametrize("seed", [0, 1])
def test_refine_random_masks(storage, seed):
    scene = si.random_scene(70 + seed, max_depth=5, sh_degree=seed + 1, storage=storage, n_prims=4)
    t = oracle.scene_tree(scene)
    L = t["leaf_key"].size
    prune, sample = si.random_masks(L, seed, p_prune=0.9, p_sample=0.05)
    c = _compare_refine(scene, prune, sample, d_cap=5, aux_width=3)
    assert c["n_pruned_groups"] > 0 and c["n_sampled"] > 0 and c["n_capped"] > 0


def test_refine_edge_cases():
    scene = si.random_scene(80, max_depth=4, sh_degree=0, storage=si.STORAGE_F32)
    L = oracle.scene_tree(scene)["leaf_key"].size
    z, o = np.zeros(L, np.uint8), np.ones(L, np.uint8)
    _compare_refine(scene, z, z, 8)            # nothing happens
    _compare_refine(scene, o, z, 8)            # every all-leaf family merged
    _compare_refine(scene, z, o, 8)            # every leaf sampled
    _compare_refine(scene, o, o, 8)            # sample marks block every merge
    _compare_refine(scene, z, o, 1)            # every sample mark capped


def test_refine_full_size():
    """Config-scale refine (2.9M leaves): top 5% sampled, bottom 20% of signal pruned."""
    import paper_2307_15333_gb300 as dot
    scene = si.nerf_synthetic_scene()
    t = oracle.scene_tree(scene)
    L = t["leaf_key"].size
    s = si.random_signal(L, 9)
    prune, sample = oracle.select(s, oracle.SELECT_FRACTION, 0.2, oracle.SELECT_FRACTION, 0.05)
    tree = _tree(scene)
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    dot.dot_select_masks(tree, torch.from_numpy(s).cuda(), dot.select_opts(2, 0.2, 2, 0.05), pm, sm)
    np.testing.assert_array_equal(pm.cpu().numpy(), prune)
    np.testing.assert_array_equal(sm.cpu().numpy(), sample)
    tree.free()
    _compare_refine(scene, prune, sample, d_cap=11)


def test_sample_by_copy_keeps_pixels_on_gpu():
    """Subdividing leaves by copy (Eq. 4) leaves the GPU render unchanged up to FP32 rounding."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(90, max_depth=5, sh_degree=2, storage=si.STORAGE_F32, n_prims=3)
    tree = _tree(scene)
    L = tree.n_leaves
    o, d = si.random_rays(3000, 3)
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    opts = dot.render_opts(eps_T=0.0)
    a = torch.empty(o.shape[0], 3, device="cuda")
    dot.dot_render_forward(tree, rays, opts, a)
    pm = torch.zeros(L, dtype=torch.uint8, device="cuda")
    sm = torch.from_numpy(si.random_masks(L, 3, 0.0, 0.5)[1]).cuda()
    counts = dot.dot_refine_plan(tree, pm, sm, 8)
    lm = torch.empty(counts["n_leaves"], dtype=torch.int32, device="cuda")
    dot.dot_refine_prune(tree, pm, sm, 8, lm)
    b = torch.empty_like(a)
    dot.dot_render_forward(tree, rays, opts, b)
    torch.testing.assert_close(b, a, rtol=2e-5, atol=2e-6)
    tree.free()


@pytest.mark.parametrize("entry", ["dot_select_masks", "dot_select_masks_noalloc"])
@pytest.mark.parametrize("D", [3, 6])
def test_select_signed_zeros_and_nan_match_oracle(entry, D):
    """Rank boundaries inside a run of mixed +0.0 / -0.0 signals, and fractions large enough to
    reach the NaNs: both selection calls give the oracle's marks bit for bit (-0 equals +0, a NaN
    comes after every number in both orders, equal keys go in leaf-id order)."""
    import paper_2307_15333_gb300 as dot
    scene = si.box_scene((-2, -2, -2), (2, 2, 2), max_depth=D, sh_degree=0)
    tree = _tree(scene)
    L = tree.n_leaves
    s = si.signed_signal(L, 40 + D)
    neg_zero = np.signbit(s) & (s == 0)
    assert neg_zero.any() and ((s == 0) & ~neg_zero).any() and np.isnan(s).any()
    sig = torch.from_numpy(s).cuda()
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    n_neg, n_pos = int((s < 0).sum()), int((s > 0).sum())
    n_num = L - int(np.isnan(s).sum())
    # bottom fraction ending inside the zeros; top fraction ending inside the zeros; NaNs reached
    f_bot = (n_neg + 0.5 * int((s == 0).sum())) / L
    f_top = (n_pos + 0.5 * int((s == 0).sum())) / L
    f_nan = (n_num + 0.5 * (L - n_num)) / L
    call = getattr(dot.dot, entry)
    for (pmode, pval, smode, sval) in [(2, f_bot, 2, f_top), (2, f_nan, 2, f_nan),
                                       (1, 0.0, 1, -0.0), (1, -0.0, 1, 0.0), (2, 1.0, 2, 0.999),
                                       (3, f_bot, 3, f_top), (3, f_nan, 3, f_nan)]:
        call(tree, sig, dot.select_opts(pmode, pval, smode, sval), pm, sm)
        rp, rs = oracle.select(s, pmode, pval, smode, sval)
        np.testing.assert_array_equal(pm.cpu().numpy(), rp)
        np.testing.assert_array_equal(sm.cpu().numpy(), rs)
    # the bottom boundary did fall among the zeros, with both signs on either side of it
    rp, _ = oracle.select(s, 2, f_bot, 0, 0.0)
    z = s == 0
    assert rp[z].any() and not rp[z].all()
    tree.free()
