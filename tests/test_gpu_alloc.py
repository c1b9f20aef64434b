"""Trees whose arrays come from a caller's dot_allocator (torch's caching allocator here)."""
import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu


def _render(dot, tree, cam_t, W, H):
    rgb = torch.empty(cam_t.shape[0] * W * H, 3, device="cuda")
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, W, H), dot.render_opts(), rgb)
    torch.cuda.synchronize()
    return rgb


def test_torch_backed_tree_renders_refines_and_frees_through_the_callbacks():
    """Build, render, refine and canonicalise a tree whose arrays are torch tensors: the images
    equal those of a library-allocated tree bit for bit, the refine allocates its new arrays and
    frees the old ones through the callbacks, and freeing the tree hands every block back."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(41, max_depth=6, sh_degree=2, storage=si.STORAGE_F16, n_prims=4)
    cams = [si.pinhole((3 * np.cos(a), 1.0, 3 * np.sin(a)), 96, 64, 90.0) for a in (0.3, 2.0)]
    cam_t = dot.cameras_tensor(cams)
    ref_tree = dot.octree_from_scene(scene)
    al = dot.dot.TorchAllocator()
    tree = dot.octree_from_scene(scene, allocator=al)
    assert al.n_alloc >= 7 and len(al.live) >= 7            # the tree's arrays
    assert torch.equal(_render(dot, tree, cam_t, 96, 64), _render(dot, ref_tree, cam_t, 96, 64))
    L = tree.n_leaves
    sig = torch.rand(L, device="cuda")
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sel = dot.select_opts(dot.dot.DOT_SELECT_FRACTION, 0.3, dot.dot.DOT_SELECT_FRACTION, 0.05)
    for t in (tree, ref_tree):
        dot.dot_select_masks(t, sig, sel, pm, sm)
        counts = dot.dot_refine_plan(t, pm, sm, 8)
        lm = torch.empty(counts["n_leaves"], dtype=torch.int32, device="cuda")
        dot.dot_refine_prune(t, pm, sm, 8, lm)
        perm = torch.empty(t.n_leaves, dtype=torch.int32, device="cuda")
        dot.dot.dot_tree_canonicalize(t, perm)
    torch.cuda.synchronize()
    assert tree.n_leaves == ref_tree.n_leaves != L
    assert al.n_free > 0                                    # the old arrays went back
    assert torch.equal(_render(dot, tree, cam_t, 96, 64), _render(dot, ref_tree, cam_t, 96, 64))
    tree.free()
    ref_tree.free()
    assert not al.live and al.n_alloc == al.n_free


def test_misaligned_blocks_fail_the_build_before_any_use():
    """An allocator whose blocks are not 16-byte aligned: each block is handed back at once and
    the build fails with DOT_ERR_OOM; nothing stays allocated."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(42, max_depth=4, sh_degree=1, storage=si.STORAGE_F32)
    al = dot.dot.TorchAllocator(offset=4)
    with pytest.raises(dot.dot.DotError) as e:
        dot.octree_from_scene(scene, allocator=al)
    assert e.value.code == dot.dot.DOT_ERR_OOM
    assert al.n_alloc >= 1 and not al.live and al.n_alloc == al.n_free
