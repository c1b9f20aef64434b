"""Canonical renumbering on the GPU (breadth-first Morton order, i.e. ascending keys) against the
oracle's sort of the keys, after refines that append cells; renders are unchanged by it."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import assert_pixels_close, oracle_side

pytestmark = pytest.mark.gpu


def _render(dot, tree, rays, R):
    out = torch.empty(R, 3, device="cuda")
    dot.dot_render_forward(tree, rays, dot.render_opts(background=(1, 1, 1), eps_T=1e-4), out)
    torch.cuda.synchronize()
    return out


def test_canonicalize_after_refines_matches_oracle():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(95, max_depth=5, sh_degree=2, storage=si.STORAGE_F16, n_prims=4)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    rng = np.random.default_rng(3)
    for r in range(3):
        L = tree.n_leaves
        pm = (rng.random(L) < 0.5).astype(np.uint8)
        sm = (rng.random(L) < 0.08).astype(np.uint8)
        tpm, tsm = torch.from_numpy(pm).cuda(), torch.from_numpy(sm).cuda()
        plan = dot.dot_refine_plan(tree, tpm, tsm, 8)
        lm = torch.empty(plan["n_leaves"], dtype=torch.int32, device="cuda")
        dot.dot_refine_prune(tree, tpm, tsm, 8, lm)
        t, _, s64, h64, _ = oracle.refine(t, s64, h64, pm, sm, 8)
    L = tree.n_leaves
    assert np.any(np.diff(t["leaf_key"].astype(np.int64)) < 0)
    # the refined tree (face-neighbour table rebuilt by each refine) renders as the oracle's
    o, d = si.random_rays(4000, 19)
    got = torch.empty(4000, 3, device="cuda")
    dot.dot_render_forward(tree, dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()),
                           dot.render_opts(background=(1, 1, 1), eps_T=1e-4), got)
    lo, size = oracle.root_of(scene)
    ref, _, _ = oracle.render(t, lo, size, s64, h64, scene.sh_degree, o, d, eps_T=1e-4)
    assert_pixels_close(got.cpu().numpy(), ref, scene.storage)
    cams = [si.pinhole((0.4, 1.1, 2.6), 640, 560, 700.0)]
    crays = dot.rays_cameras(dot.cameras_tensor(cams), 640, 560)
    o, d = si.random_rays(5000, 17)
    brays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    before_c, before_b = _render(dot, tree, crays, 640 * 560), _render(dot, tree, brays, 5000)
    pre = tree.export()
    aux = torch.from_numpy(rng.normal(size=(L, 3)).astype(np.float32)).cuda()
    aux_out = torch.empty_like(aux)
    perm = torch.empty(L, dtype=torch.int32, device="cuda")
    dot.dot.dot_tree_canonicalize(tree, perm, [(aux, aux_out)])
    nt, operm, (os64, oh64) = oracle.canonicalize(t, (s64, h64))
    ex = tree.export()
    for key in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        assert np.array_equal(ex[key], nt[key]), key
    p = perm.cpu().numpy()
    np.testing.assert_array_equal(p, operm)
    np.testing.assert_array_equal(ex["sigma"], pre["sigma"][p])
    np.testing.assert_array_equal(ex["sh"], pre["sh"][p])
    np.testing.assert_array_equal(aux_out.cpu().numpy(), aux.cpu().numpy()[p])
    np.testing.assert_allclose(si.storage_to_f64(ex["sigma"], scene.storage), os64,
                               rtol=2e-3, atol=1e-3)
    assert torch.equal(_render(dot, tree, crays, 640 * 560), before_c)
    assert torch.equal(_render(dot, tree, brays, 5000), before_b)
    assert tree.status() == 0
    tree.free()


def test_canonicalize_built_and_compressed_tree_is_identity():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(96, max_depth=5, sh_degree=1, storage=si.STORAGE_BF16, n_prims=3)
    tree = dot.octree_from_scene(scene)
    dot.dot.dot_compress_sh(tree, 6)
    o, d = si.random_rays(2000, 18)
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    before = _render(dot, tree, rays, 2000)
    pre = tree.export()
    perm = torch.empty(tree.n_leaves, dtype=torch.int32, device="cuda")
    dot.dot.dot_tree_canonicalize(tree, perm)
    assert np.array_equal(perm.cpu().numpy(), np.arange(tree.n_leaves))
    ex = tree.export()
    for key in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key", "sigma", "sh"):
        assert np.array_equal(ex[key], pre[key]), key
    assert tree.palette_bits == 6
    assert torch.equal(_render(dot, tree, rays, 2000), before)
    tree.free()
