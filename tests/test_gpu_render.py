"""GPU forward render (Eq. 1-2) vs the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import assert_pixels_close, oracle_side

pytestmark = pytest.mark.gpu


def _gpu_render(tree, o, d, **kw):
    import paper_2307_15333_gb300 as dot
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    R = o.shape[0]
    rgb = torch.empty(R, 3, device="cuda")
    T = torch.empty(R, device="cuda")
    dot.dot_render_forward(tree, rays, dot.render_opts(**kw), rgb, T)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), T.cpu().numpy()


def test_tiny_config_camera_mode_matches_buffer_mode_and_oracle():
    import paper_2307_15333_gb300 as dot
    scene, cams = si.config_tiny()
    tree = dot.octree_from_scene(scene)
    cam_t = dot.cameras_tensor(cams)
    rgb_c = torch.empty(64 * 64, 3, device="cuda")
    T_c = torch.empty(64 * 64, device="cuda")
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 64, 64), opts, rgb_c, T_c)
    o, d = si.camera_rays(cams[0])
    rgb_b, T_b = _gpu_render(tree, o, d, background=(1, 1, 1), eps_T=1e-4)
    # in-kernel ray generation follows the same float32 operations as the input generator
    np.testing.assert_array_equal(rgb_c.cpu().numpy(), rgb_b)
    np.testing.assert_array_equal(T_c.cpu().numpy(), T_b)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    ref, Tref, _ = oracle.render(t, lo, size, s64, h64, scene.sh_degree, o, d, eps_T=1e-4)
    assert_pixels_close(rgb_b, ref, scene.storage)
    assert_pixels_close(T_b, Tref, scene.storage, what="T")
    assert (ref.min() < 0.9) and np.any(Tref < 1e-3)     # the sphere is in view and opaque
    tree.free()


CASES = [(st, deg) for st in (si.STORAGE_F32, si.STORAGE_F16, si.STORAGE_BF16) for deg in range(4)]


@pytest.mark.parametrize("storage,deg", CASES)
def test_random_scene_random_rays(storage, deg):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(10 + deg, max_depth=6, sh_degree=deg, storage=storage, n_prims=4)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(3000, 100 + deg)
    for eps in (1e-4, 0.0):
        for act in (dot.dot.DOT_ACT_SIGMOID, dot.dot.DOT_ACT_LINEAR):
            bg = (0.2, 0.5, 1.0)
            got, Tg = _gpu_render(tree, o, d, background=bg, eps_T=eps, color_act=act)
            ref, Tr, _ = oracle.render(t, lo, size, s64, h64, deg, o, d, bg=bg, eps_T=eps,
                                       color_act=act)
            assert_pixels_close(got, ref, storage)
            assert_pixels_close(Tg, Tr, storage, what="T")
    tree.free()


@pytest.mark.parametrize("precision", [1, 2])
def test_precision_modes_on_fp32(precision):
    """Fast plane times stay within the 16-bit-leaf tolerance on FP32 leaves; exact mode meets
    the FP32 tolerance."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(31, max_depth=7, sh_degree=2, storage=si.STORAGE_F32, n_prims=5)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(4000, 7)
    got, _ = _gpu_render(tree, o, d, precision=precision)
    ref, _, _ = oracle.render(t, lo, size, s64, h64, 2, o, d)
    assert_pixels_close(got, ref, si.STORAGE_F32, exact=(precision == 2))
    tree.free()


def test_edge_cases():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(5, max_depth=5, sh_degree=1, storage=si.STORAGE_F32)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    # no rays
    got, _ = _gpu_render(tree, np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    assert got.shape == (0, 3)
    # rays that miss the root, rays starting inside it, exactly axis-aligned rays through cell
    # faces and centres, and a ray along a root edge
    o = np.array([[3, 3, 3], [0, 0, 0], [0.1, -0.2, 0.3], [0.0, 0.0, 5.0], [0.125, 0.375, -5.0],
                  [-1.0, -1.0, 5.0], [0.03125, 0.0, 0.0]], np.float32)
    d = np.array([[1, 0, 0], [0, 0, 1], [0.6, 0.0, -0.8], [0, 0, -1], [0, 0, 1], [0, 0, -1],
                  [0, 1, 0]], np.float32)
    got, Tg = _gpu_render(tree, o, d, background=(0.3, 0.6, 0.9))
    ref, Tr, _ = oracle.render(t, lo, size, s64, h64, 1, o, d, bg=(0.3, 0.6, 0.9))
    np.testing.assert_array_equal(got[0], np.float32([0.3, 0.6, 0.9]))
    assert Tg[0] == 1.0
    assert_pixels_close(got, ref, si.STORAGE_F32)
    tree.free()


def _edge_rays(t, s64, lo, size, n_leaves=4):
    """Rays that miss the root, start inside it, run along root edges and faces, and, for a few
    occupied leaves: along the leaf's edge (two exit planes tied all the way), along one of its
    faces and through its centre on each axis, and through its corner on the two diagonals
    (three planes tied at every lattice corner)."""
    o = [[3, 3, 3], [0, 0, 0], [0.1, -0.2, 0.3], [-1.0, -1.0, 5.0], [0.03125, 0.0, 0.0],
         [-1.0, 0.1, 5.0], [1.0, 0.2, -5.0]]
    d = [[1, 0, 0], [0, 0, 1], [0.6, 0.0, -0.8], [0, 0, -1], [0, 1, 0], [0, 0, -1], [0, 0, 1]]
    keys = np.asarray(t["leaf_key"], np.uint64)
    occ = np.nonzero(s64 > 0)[0]
    for v in occ[:: max(1, len(occ) // n_leaves)][:n_leaves]:
        k = int(keys[v])
        lv = (k.bit_length() - 1) // 3
        c = [0, 0, 0]
        for i in range(lv):
            tri = (k >> (3 * (lv - 1 - i))) & 7
            c = [(c[0] << 1) | (tri >> 2), (c[1] << 1) | ((tri >> 1) & 1), (c[2] << 1) | (tri & 1)]
        cs = size / (1 << lv)
        x0, y0, z0 = (lo[a] + c[a] * cs for a in range(3))
        xc, yc, zc = x0 + cs / 2, y0 + cs / 2, z0 + cs / 2
        o += [[x0, y0, 5.0], [-5.0, y0, zc], [xc, 5.0, zc], [xc, yc, -5.0],
              [x0 - 3.0, y0 - 3.0, z0 - 3.0], [x0 + 3.0, y0 + 3.0, z0 - 3.0]]
        d += [[0, 0, -1], [1, 0, 0], [0, -1, 0], [0, 0, 1], [1, 1, 1], [-1, -1, 1]]
    o = np.array(o, np.float32)
    d = np.array(d, np.float32)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d


@pytest.mark.parametrize("storage", [si.STORAGE_F32, si.STORAGE_F16])
def test_fast_path_edge_cases(storage):
    """The fast (float32 plane time) march on the edge-case rays, in a small launch and in the
    large-launch build (the rays tiled past two full waves): both match the oracle at the
    fast-mode tolerance and equal each other bit for bit."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(5, max_depth=5, sh_degree=3, storage=storage)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = _edge_rays(t, s64, lo, size)
    small, Ts = _gpu_render(tree, o, d, background=(0.3, 0.6, 0.9), precision=1)
    ref, Tr, _ = oracle.render(t, lo, size, s64, h64, 3, o, d, bg=(0.3, 0.6, 0.9))
    np.testing.assert_array_equal(small[0], np.float32([0.3, 0.6, 0.9]))
    assert_pixels_close(small, ref, storage, exact=False)
    assert_pixels_close(Ts, Tr, storage, exact=False, what="T")
    reps = (2 * 1024 * 152) // o.shape[0] + 1
    big, Tb = _gpu_render(tree, np.tile(o, (reps, 1)), np.tile(d, (reps, 1)),
                          background=(0.3, 0.6, 0.9), precision=1)
    assert np.array_equal(big, np.tile(small, (reps, 1))), "large launch differs from small"
    assert np.array_equal(Tb, np.tile(Ts, reps)), "large launch T differs from small"
    assert tree.status() == 0
    tree.free()


def test_full_size_nerf_synthetic_sampled_pixels():
    """Config at full size (2.9M leaves, 800x800 views) in the bench's launch configuration
    (camera mode, all views in one launch, nearest-neighbour view order); sampled pixels against
    the oracle."""
    import paper_2307_15333_gb300 as dot
    scene, cams = si.config_nerf_synthetic(n_views=100)
    tree = dot.octree_from_scene(scene)
    cam_t = dot.cameras_tensor(cams)
    order = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    R = 100 * 800 * 800
    rgb = torch.empty(R, 3, device="cuda")
    opts = dot.render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4)
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 800, 800, order), opts, rgb)
    torch.cuda.synchronize()
    assert tree.status() == 0
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    rng = np.random.default_rng(3)
    for v in (0, 37, 99):
        pix = rng.integers(0, 800 * 800, 1500)
        o, d = si.camera_rays(cams[v], pix)
        ref, _, _ = oracle.render(t, lo, size, s64, h64, 3, o, d)
        got = rgb[v * 800 * 800 + torch.from_numpy(pix).cuda()].cpu().numpy()
        assert_pixels_close(got, ref, scene.storage)
        assert np.std(ref) > 0.05                       # not a blank view
    tree.free()


def test_full_size_tanks_temples_sampled_pixels():
    import paper_2307_15333_gb300 as dot
    scene, cams = si.config_tanks_temples(n_views=6)
    tree = dot.octree_from_scene(scene)
    cam_t = dot.cameras_tensor(cams)
    order = torch.from_numpy(dot.dot.dot_camera_order(cam_t.cpu().numpy())).cuda()
    R = 6 * 1920 * 1080
    rgb = torch.empty(R, 3, device="cuda")
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 1920, 1080, order), dot.render_opts(), rgb)
    torch.cuda.synchronize()
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    rng = np.random.default_rng(4)
    for v in (0, 5):
        pix = rng.integers(0, 1920 * 1080, 1500)
        o, d = si.camera_rays(cams[v], pix)
        ref, _, _ = oracle.render(t, lo, size, s64, h64, 3, o, d)
        got = rgb[v * 1920 * 1080 + torch.from_numpy(pix).cuda()].cpu().numpy()
        assert_pixels_close(got, ref, scene.storage)
    tree.free()


def test_step_cap_sets_status_without_hanging():
    """A per-ray step cap that is too small truncates rays and raises the status bit."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(6, max_depth=6, sh_degree=0, storage=si.STORAGE_F32)
    tree = dot.octree_from_scene(scene)
    o, d = si.random_rays(500, 1)
    _gpu_render(tree, o, d, max_steps=2)
    assert tree.status() & dot.dot.DOT_STATUS_STEP_LIMIT
    assert tree.status() == 0                          # read clears it
    _gpu_render(tree, o, d)
    assert tree.status() == 0
    tree.free()


def test_view_order_renders_the_same_rays():
    """A view order changes only the schedule: the images are identical bit for bit; an order
    entry out of range skips its views and sets DOT_STATUS_BAD_INPUT."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(12, max_depth=5, sh_degree=2, storage=si.STORAGE_F16, n_prims=4)
    tree = dot.octree_from_scene(scene)
    cams = [si.pinhole((3 * np.cos(a), 1.0, 3 * np.sin(a)), 320, 240, 300.0)
            for a in np.linspace(0, 6, 7)]
    recs = np.stack([c.packed() for c in cams])
    cam_t = dot.cameras_tensor(cams)
    R = 7 * 320 * 240
    opts = dot.render_opts(background=(1, 1, 1))
    a = torch.empty(R, 3, device="cuda")
    b = torch.full((R, 3), -1.0, device="cuda")
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 320, 240), opts, a)
    order = torch.from_numpy(dot.dot.dot_camera_order(recs)).cuda()
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 320, 240, order), opts, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert tree.status() == 0
    bad = order.clone()
    bad[3] = 7
    c = torch.full((R, 3), -1.0, device="cuda")
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, 320, 240, bad), opts, c)
    torch.cuda.synchronize()
    assert tree.status() == dot.dot.DOT_STATUS_BAD_INPUT
    skipped = int(order[3])
    img = c.view(7, 240 * 320, 3)
    assert (img[skipped] == -1.0).all()
    others = [v for v in range(7) if v != skipped]
    assert torch.equal(img[others], a.view(7, -1, 3)[others])
    tree.free()


def _forward_all(dot, tree, cam_t, W, H, opts):
    n = cam_t.shape[0]
    rgb = torch.empty(n * W * H, 3, device="cuda")
    T = torch.empty(n * W * H, device="cuda")
    dot.dot_render_forward(tree, dot.rays_cameras(cam_t, W, H), opts, rgb, T)
    torch.cuda.synchronize()
    return rgb.cpu(), T.cpu()


def test_views_to_host_match_the_device_forward():
    """dot_render_views_host writes the same bits as one dot_render_forward launch, both ways:
    into pinned (mapped) host buffers by one launch writing in place, and into pageable ones
    through chunks of about 2^23 rays over two render streams, three chunk buffers in a ring and
    copies on a third stream (40 views of 800x800 go in seven chunks: 10, 10, 10, 5, 3, 1, 1
    views, so the ring wraps); with and without a view order and T; a given workspace is
    reused."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(21, max_depth=6, sh_degree=3, storage=si.STORAGE_F16, n_prims=5)
    tree = dot.octree_from_scene(scene)
    W, H, n = 800, 800, 40
    cams = [si.pinhole((3 * np.cos(a), 0.5 + 0.3 * np.sin(3 * a), 3 * np.sin(a)), W, H, 700.0)
            for a in np.linspace(0, 6.2, n)]
    recs = torch.from_numpy(np.stack([c.packed() for c in cams]).astype(np.float32))
    opts = dot.render_opts(background=(1, 1, 1))
    ref, Tref = _forward_all(dot, tree, recs.cuda(), W, H, opts)
    ref = ref.view(n, H, W, 3)
    Tref = Tref.view(n, H, W)
    order = dot.dot.dot_camera_order(recs.numpy())
    ws = torch.empty(dot.dot.dot_render_views_host_workspace(n, W, H, True), dtype=torch.uint8,
                     device="cuda")
    # (pinned images, view order, T wanted, pinned T): a pageable T sends both through the copies
    for pinned, view_order, with_T, pinned_T in ((True, order, True, True), (False, None, False, False),
                                                 (True, None, True, True), (False, order, False, False),
                                                 (True, order, True, False)):
        out = torch.full((n, H, W, 3), -1.0, pin_memory=pinned)
        T = torch.full((n, H, W), -1.0, pin_memory=pinned_T) if with_T else None
        dot.dot.dot_render_views_host(tree, recs, W, H, opts, out, T_host=T,
                                      view_order=view_order, workspace=ws)
        assert torch.equal(out, ref)
        if with_T:
            assert torch.equal(T, Tref)
    # the application call (pinned output, nearest-neighbour order)
    from paper_2307_15333_gb300.render import render_views
    assert torch.equal(render_views(tree, recs, W, H, opts), ref)
    assert tree.status() == 0
    tree.free()


def test_views_to_host_argument_errors():
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(22, max_depth=4, sh_degree=1, storage=si.STORAGE_F32)
    tree = dot.octree_from_scene(scene)
    cams = [si.pinhole((0.0, 0.0, 3.0 + i), 64, 48, 60.0) for i in range(5)]
    recs = torch.from_numpy(np.stack([c.packed() for c in cams]).astype(np.float32))
    out = torch.zeros(5, 48, 64, 3)
    opts = dot.render_opts()
    for bad in (np.array([0, 1, 2, 3, 3], np.int32), np.array([0, 1, 2, 3, 5], np.int32),
                np.array([0, 1, 2, 3, -1], np.int32)):
        with pytest.raises(dot.dot.DotError) as e:
            dot.dot.dot_render_views_host(tree, recs, 64, 48, opts, out, view_order=bad)
        assert e.value.code == dot.dot.DOT_ERR_INVALID_ARG and "permutation" in str(e.value)
    need = dot.dot.dot_render_views_host_workspace(5, 64, 48)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(dot.dot.DotError) as e:
        dot.dot.dot_render_views_host(tree, recs, 64, 48, opts, out, workspace=small)
    assert "workspace" in str(e.value)
    sig = dot.render_opts(signal_mode=dot.dot.DOT_SIGNAL_MAX_WEIGHT)
    with pytest.raises(dot.dot.DotError):
        dot.dot.dot_render_views_host(tree, recs, 64, 48, sig, out)
    assert (out == 0).all()                            # nothing was rendered or copied
    # no views: nothing to do
    dot.dot.dot_render_views_host(tree, recs[:0], 64, 48, opts, torch.zeros(0))
    tree.free()


@pytest.mark.parametrize("depth,radius,storage", [(12, 0.01, si.STORAGE_F32), (12, 0.01, si.STORAGE_F16),
                                                  (16, 0.0006, si.STORAGE_F32)])
def test_deep_tree_matches_oracle(depth, radius, storage):
    """Trees down to the finest level (16): a small sphere and box carved deep, so that rays near
    them cross neighbours up to 15 levels apart; rays aimed at the primitives."""
    import paper_2307_15333_gb300 as dot
    c = np.array([0.1, -0.05, 0.02])
    prims = si._prims([si.sphere(tuple(c), radius, (0.0, 0.0, 0.0), 1.0),
                       si.box(tuple(c - [2 * radius, radius, 0.5 * radius]),
                              tuple(c + [-0.5 * radius, 2 * radius, 2 * radius]), (0.0, 0.0, 0.0), 1.0)])
    scene = si.Scene(f"deep{depth}", (0.0, 0.0, 0.0), 1.0, depth, 1, storage, prims,
                     5.0 / radius, 50.0 / radius, 0.4, 0.2, 41)
    tree = dot.octree_from_scene(scene)
    assert tree.info().max_level == depth
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    rng = np.random.default_rng(depth)
    u = rng.normal(size=(3000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    o = (c + 3.0 * u).astype(np.float32)
    aim = c + rng.uniform(-3 * radius, 3 * radius, size=(3000, 3))
    d = aim - o.astype(np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    got, Tg = _gpu_render(tree, o, d)
    ref, Tr, _ = oracle.render(t, lo, size, s64, h64, 1, o, d)
    assert_pixels_close(got, ref, storage)
    assert_pixels_close(Tg, Tr, storage, what="T")
    assert np.mean(Tr < 0.5) > 0.2                     # many rays do hit the primitives
    assert tree.status() == 0
    tree.free()
