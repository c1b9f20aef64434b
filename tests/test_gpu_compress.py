"""Compressed models (Sec. 4.1) on the GPU: the median-cut palette and indices against the
oracle's quantiser, renders of a compressed tree against the oracle's render of the expanded
coefficients, and the calls a compressed tree refuses."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import ABS16, oracle_side

pytestmark = pytest.mark.gpu


def _spacing(x, storage):
    x = np.abs(np.asarray(x, np.float64))
    if storage == si.STORAGE_F16:
        return np.spacing(x.astype(np.float16)).astype(np.float64)
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 2.0 ** (e - 7)


CASES = [(st, deg, bits) for st in (si.STORAGE_F16, si.STORAGE_BF16) for deg, bits in
         ((1, 4), (2, 8), (3, 10))]


@pytest.mark.parametrize("storage,deg,bits", CASES)
def test_palette_and_render_match_oracle(storage, deg, bits):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(80 + deg, max_depth=6, sh_degree=deg, storage=storage, n_prims=4)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    L, K = s64.size, (deg + 1) ** 2
    idx_ref, pal_ref = oracle.median_cut(h64.reshape(L, 3 * K), bits)
    dot.dot.dot_compress_sh(tree, bits)
    assert tree.palette_bits == bits
    idx = tree.palette_index.cpu().numpy()
    np.testing.assert_array_equal(idx, idx_ref)
    pal = tree.palette.float().cpu().numpy().astype(np.float64).reshape(1 << bits, 3 * K)
    assert (np.abs(pal - pal_ref) <= _spacing(pal_ref, storage)).all()
    # export writes the expanded coefficients; densities are untouched
    ex = tree.export()
    np.testing.assert_array_equal(si.storage_to_f64(ex["sigma"], storage), s64)
    np.testing.assert_array_equal(si.storage_to_f64(ex["sh"], storage).reshape(L, -1), pal[idx])
    # the compressed render is the render of the expanded coefficients
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(3000, 500 + deg)
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    opts = dot.render_opts(background=(0.2, 0.5, 0.9), eps_T=1e-4)
    rgb = torch.empty(3000, 3, device="cuda")
    dot.dot_render_forward(tree, rays, opts, rgb)
    torch.cuda.synchronize()
    ref, _, _ = oracle.render(t, lo, size, s64, pal[idx].reshape(L, 3, K), deg, o, d,
                              bg=(0.2, 0.5, 0.9), eps_T=1e-4)
    assert np.abs(rgb.cpu().numpy() - ref).max() <= ABS16
    assert tree.status() == 0
    tree.free()


def test_compressed_camera_render_and_signal():
    """Camera rays through the large-launch build and the density-only signal on a compressed
    tree equal the uncompressed tree's when the palette holds every row (2^bits >= L)."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(91, max_depth=5, sh_degree=3, storage=si.STORAGE_F16, n_prims=3)
    a = dot.octree_from_scene(scene)
    b = dot.octree_from_scene(scene)
    L = a.n_leaves
    bits = int(np.ceil(np.log2(L)))
    assert bits <= 16
    dot.dot.dot_compress_sh(b, bits)
    cams = [si.pinhole((0.3, 0.8, 3.0), 700, 600, 800.0), si.pinhole((-2.5, 0.2, 1.5), 700, 600, 700.0)]
    rays = dot.rays_cameras(dot.cameras_tensor(cams), 700, 600)
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    ra = torch.empty(2 * 700 * 600, 3, device="cuda")
    rb = torch.empty_like(ra)
    dot.dot_render_forward(a, rays, opts, ra)
    dot.dot_render_forward(b, rays, opts, rb)
    sa = torch.zeros(L, device="cuda")
    sb = torch.zeros(L, device="cuda")
    dot.dot_accumulate_signal(a, rays, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, sa)
    dot.dot_accumulate_signal(b, rays, opts, dot.dot.DOT_SIGNAL_MAX_WEIGHT, sb)
    torch.cuda.synchronize()
    assert torch.equal(ra, rb)
    assert torch.equal(sa, sb)
    a.free()
    b.free()


def test_compressed_tree_refuses_training_and_refine():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(92, max_depth=4, sh_degree=1, storage=si.STORAGE_BF16, n_prims=2)
    tree = dot.octree_from_scene(scene)
    dot.dot.dot_compress_sh(tree, 3)
    L, K = tree.n_leaves, 4
    o, d = si.random_rays(10, 1)
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    opts = dot.render_opts()
    z = lambda *s: torch.zeros(*s, device="cuda")
    with pytest.raises(dot.DotError) as e:
        dot.dot_render_backward(tree, rays, opts, z(10, 3), z(10, 3), z(L), z(L, 3, K))
    assert e.value.code == dot.dot.DOT_ERR_UNSUPPORTED
    with pytest.raises(dot.DotError) as e:
        dot.dot.dot_rmsprop_step(tree, z(L), z(L, 3, K), z(L), z(L, 3, K), dot.dot.rmsprop_opts())
    assert e.value.code == dot.dot.DOT_ERR_UNSUPPORTED
    m = torch.zeros(L, dtype=torch.uint8, device="cuda")
    with pytest.raises(dot.DotError) as e:
        dot.dot_refine_plan(tree, m, m, 8)
    assert e.value.code == dot.dot.DOT_ERR_UNSUPPORTED
    with pytest.raises(dot.DotError) as e:
        dot.dot.dot_compress_sh(tree, 3)
    assert e.value.code == dot.dot.DOT_ERR_UNSUPPORTED
    f32 = dot.octree_from_scene(si.random_scene(93, max_depth=3, sh_degree=1, n_prims=2))
    with pytest.raises(dot.DotError) as e:
        dot.dot.dot_compress_sh(f32, 4)
    assert e.value.code == dot.dot.DOT_ERR_UNSUPPORTED
    tree.free()
    f32.free()


def test_slot_tables_serve_compressed_trees():
    """Requests on compressed trees through one slot-table launch equal plain forward renders,
    and a table mixing compressed and uncompressed trees is refused."""
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    trees = [dot.octree_from_scene(si.random_scene(97 + i, max_depth=5, sh_degree=3,
                                                   storage=si.STORAGE_F16, n_prims=3))
             for i in range(2)]
    for t in trees:
        dot.dot.dot_compress_sh(t, 8)
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    rng = np.random.default_rng(0)
    reqs = []
    for i, (w, h) in enumerate([(64, 48), (200, 120), (33, 77)]):
        pos = 3.0 * np.array([rng.uniform(-1, 1), rng.uniform(0.2, 1), rng.uniform(-1, 1)])
        reqs.append(serve.Request(i, i % 2, w, h, si.pinhole(pos, w, h, 1.2 * w).packed(), 0.0))
    srv = serve.BatchedServer(trees, opts, pool_floats=4 << 20, max_slots=8)
    mixed, alone = srv.render_alone_and_mixed(reqs)
    for r, m, a in zip(reqs, mixed, alone):
        assert torch.equal(m, a)
        ref = torch.empty(r.width * r.height, 3, device="cuda")
        cam = torch.from_numpy(r.camera).cuda().view(1, 18)
        dot.dot_render_forward(trees[r.tree], dot.rays_cameras(cam, r.width, r.height), opts, ref)
        torch.cuda.synchronize()
        assert torch.equal(m.view(-1, 3), ref)
    plain = dot.octree_from_scene(si.random_scene(99, max_depth=4, sh_degree=3,
                                                  storage=si.STORAGE_F16, n_prims=2))
    table = torch.zeros(16 + 96 * 4, dtype=torch.uint8, device="cuda")
    counter = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(dot.DotError):
        dot.dot.dot_render_slots([trees[0], plain], table, 4, opts, counter)
    for t in trees + [plain]:
        t.free()


def test_full_size_compressed_model_matches_oracle():
    """The bench's compressed model at full size: 2.9 M-leaf tree, 2^16-row palette.  Palette
    indices bit-exact against the oracle's median cut; sampled pixels of view-ordered 800x800
    camera renders (the bench's launch configuration) against the oracle's render of the
    palette rows."""
    import paper_2307_15333_gb300 as dot
    scene, cams = si.config_nerf_synthetic(n_views=100)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    L, K = s64.size, scene.n_coeffs
    idx_ref, pal_ref = oracle.median_cut(h64.reshape(L, 3 * K), 16)
    dot.dot.dot_compress_sh(tree, 16)
    idx = tree.palette_index.cpu().numpy()
    np.testing.assert_array_equal(idx, idx_ref)
    pal = tree.palette.float().cpu().numpy().astype(np.float64).reshape(1 << 16, 3 * K)
    assert (np.abs(pal - pal_ref) <= _spacing(pal_ref, scene.storage)).all()
    cam_t = dot.cameras_tensor(cams)
    order = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    rgb = torch.empty(100 * 800 * 800, 3, device="cuda")
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 800, 800, order), opts, rgb)
    torch.cuda.synchronize()
    assert tree.status() == 0
    lo, size = oracle.root_of(scene)
    rows = pal[idx].reshape(L, 3, K)
    rng = np.random.default_rng(6)
    for v in (0, 61):
        pix = rng.integers(0, 800 * 800, 1500)
        o, d = si.camera_rays(cams[v], pix)
        ref, _, _ = oracle.render(t, lo, size, s64, rows, 3, o, d)
        got = rgb[v * 800 * 800 + torch.from_numpy(pix).cuda()].cpu().numpy()
        assert np.abs(got - ref).max() <= ABS16
    tree.free()
