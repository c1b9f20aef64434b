"""GPU backward (recompute-the-march) and the fused / standalone training signal vs the oracle."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import assert_sums_close, assert_sums_close_grazing, oracle_side

pytestmark = pytest.mark.gpu


def _rays(o, d):
    import paper_2307_15333_gb300 as dot
    return dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())


CASES = [(st, deg) for st in (si.STORAGE_F32, si.STORAGE_F16, si.STORAGE_BF16) for deg in range(4)]


@pytest.mark.parametrize("storage,deg", CASES)
def test_backward_matches_oracle(storage, deg):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(40 + deg, max_depth=5, sh_degree=deg, storage=storage, n_prims=4)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(4000, 200 + deg)
    # early termination is a discrete decision taken on T: rays whose FP64 transmittance comes
    # within 0.1% of eps_T may stop one segment apart in FP32, so they are set aside (rarely any)
    _, _, _, margin = oracle.render(t, lo, size, s64, h64, deg, o, d, bg=(0.1, 0.7, 0.4),
                                    eps_T=1e-4, margin=True)
    keep = margin > 1e-3
    assert keep.mean() > 0.99
    o, d = np.ascontiguousarray(o[keep]), np.ascontiguousarray(d[keep])
    R = o.shape[0]
    g = np.random.default_rng(deg).normal(size=(R, 3)).astype(np.float32)
    rays = _rays(o, d)
    opts = dot.render_opts(background=(0.1, 0.7, 0.4), eps_T=1e-4)
    rgb = torch.empty(R, 3, device="cuda")
    dot.dot_render_forward(tree, rays, opts, rgb)
    L, K = tree.n_leaves, (deg + 1) ** 2
    gs = torch.zeros(L, device="cuda")
    gsh = torch.zeros(L, 3, K, device="cuda")
    sig = torch.zeros(L, device="cuda")
    opts_s = dot.render_opts(background=(0.1, 0.7, 0.4), eps_T=1e-4,
                             signal_mode=dot.dot.DOT_SIGNAL_SUM_ALPHA)
    dot.dot_render_backward(tree, rays, opts_s, torch.from_numpy(g).cuda(), rgb, gs, gsh, sig)
    torch.cuda.synchronize()
    rs, rsh, asg, ash = oracle.backward(t, lo, size, s64, h64, deg, o, d, g.astype(np.float64),
                                        bg=(0.1, 0.7, 0.4), eps_T=1e-4)
    # FP32 leaves (exact mode): 1e-5 of the summed magnitudes; 16-bit leaves (fast mode):
    # 2e-3 of the summed magnitudes plus 1e-5 absolute (grazing rays move a boundary by ~1e-7)
    rel, floor = (1e-5, 1e-7) if storage == si.STORAGE_F32 else (2e-3, 1e-5)
    assert np.abs(rs).max() > 0
    assert_sums_close(gs.cpu().numpy(), rs, asg, rel, "dsigma", floor)
    assert_sums_close(gsh.cpu().numpy(), rsh, ash, rel, "dsh", floor)
    S = np.zeros(L)
    oracle.render(t, lo, size, s64, h64, deg, o, d, eps_T=1e-4, signal=S,
                  signal_mode=oracle.SIGNAL_SUM_ALPHA)
    assert_sums_close(sig.cpu().numpy(), S, S, rel, "signal", floor)
    tree.free()


def test_autograd_function_delivers_fp32_gradients():
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import autograd
    scene = si.random_scene(50, max_depth=5, sh_degree=3, storage=si.STORAGE_F16, n_prims=3)
    tree = dot.octree_from_scene(scene)
    o, d = si.random_rays(2000, 9)
    rays = _rays(o, d)
    opts = dot.render_opts()
    sinks = autograd.gradient_sinks(tree)
    rgb = autograd.render(tree, rays, opts, sinks)
    target = torch.rand_like(rgb)
    loss = ((rgb - target) ** 2).sum()
    loss.backward()
    assert sinks[0].grad.dtype == torch.float32 and sinks[1].grad.shape == (tree.n_leaves, 3, 16)
    # same as calling the entry point directly with dL/drgb = 2 (rgb - target)
    gs = torch.zeros_like(sinks[0])
    gsh = torch.zeros_like(sinks[1])
    dot.dot_render_backward(tree, rays, opts, (2 * (rgb - target)).detach().contiguous(),
                            rgb.detach().contiguous(), gs, gsh)
    torch.testing.assert_close(sinks[0].grad, gs, rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(sinks[1].grad, gsh, rtol=1e-5, atol=1e-6)
    tree.free()


@pytest.mark.parametrize("mode", ["sum_alpha", "max_weight", "sigma"])
def test_accumulate_signal(mode):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(60, max_depth=6, sh_degree=1, storage=si.STORAGE_F32, n_prims=4)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(5000, 61)
    L = tree.n_leaves
    sig = torch.zeros(L, device="cuda")
    m = {"sum_alpha": dot.dot.DOT_SIGNAL_SUM_ALPHA, "max_weight": dot.dot.DOT_SIGNAL_MAX_WEIGHT,
         "sigma": dot.dot.DOT_SIGNAL_SIGMA}[mode]
    dot.dot_accumulate_signal(tree, _rays(o, d), dot.render_opts(), m, sig)
    torch.cuda.synchronize()
    got = sig.cpu().numpy()
    if mode == "sigma":
        np.testing.assert_array_equal(got, np.maximum(s64, 0).astype(np.float32))
    else:
        S = np.zeros(L)
        oracle.render(t, lo, size, s64, h64, 1, o, d, signal=S,
                      signal_mode=oracle.SIGNAL_SUM_ALPHA if mode == "sum_alpha" else oracle.SIGNAL_MAX_WEIGHT)
        assert_sums_close(got, S, S, 1e-5, mode)
        assert (S > 0).sum() > 50
        if mode == "sum_alpha":
            # the fused signal of the forward equals the standalone one bit for bit
            sig2 = torch.zeros(L, device="cuda")
            rgb = torch.empty(o.shape[0], 3, device="cuda")
            dot.dot_render_forward(tree, _rays(o, d), dot.render_opts(signal_mode=m), rgb, None, sig2)
            torch.testing.assert_close(sig2, sig, rtol=1e-6, atol=1e-6)
    tree.free()


def test_large_backward_launch_equals_small_launches():
    """A backward over 400 k camera rays (the occupancy build for launches of two full waves)
    gives the gradients of the same rays run as small buffer launches (the build the oracle
    parity tests cover), up to the order of the FP32 atomic sums."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(44, max_depth=6, sh_degree=3, storage=si.STORAGE_F16, n_prims=4)
    tree = dot.octree_from_scene(scene)
    cams = [si.pinhole((0.2, 0.9, 2.8), 640, 640, 700.0)]
    R = 640 * 640
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    rays = dot.rays_cameras(dot.cameras_tensor(cams), 640, 640)
    rgb = torch.empty(R, 3, device="cuda")
    dot.dot_render_forward(tree, rays, opts, rgb)
    g = torch.from_numpy(np.random.default_rng(4).normal(0, 1e-2, (R, 3)).astype(np.float32)).cuda()
    L, K = tree.n_leaves, 16
    gs_a, gsh_a = torch.zeros(L, device="cuda"), torch.zeros(L, 3, K, device="cuda")
    dot.dot_render_backward(tree, rays, opts, g, rgb, gs_a, gsh_a)
    o, d = si.camera_rays(cams[0])
    gs_b, gsh_b = torch.zeros(L, device="cuda"), torch.zeros(L, 3, K, device="cuda")
    step = 100_000                      # below the two-wave threshold: the small-launch build
    for s in range(0, R, step):
        e = min(R, s + step)
        rb = dot.rays_buffer(torch.from_numpy(o[s:e]).cuda(), torch.from_numpy(d[s:e]).cuda())
        dot.dot_render_backward(tree, rb, opts, g[s:e].contiguous(), rgb[s:e].contiguous(), gs_b, gsh_b)
    torch.cuda.synchronize()
    for a, b in ((gs_a, gs_b), (gsh_a, gsh_b)):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        scale = np.abs(a).max()
        assert scale > 0
        assert np.abs(a - b).max() <= 1e-5 * scale + 1e-9
    assert tree.status() == 0
    tree.free()


def _separate_and_fused(dot, tree, rays, opts_sig, tgt, R, L, K):
    """The three separate calls (forward with signal, MSE gradient, backward) and the fused pass
    on the same rays; returns both sets of outputs."""
    plain = dot.render_opts(background=tuple(opts_sig.background), eps_T=opts_sig.eps_T)
    z = lambda *s: torch.zeros(*s, device="cuda")
    a = dict(rgb=z(R, 3), g=z(R, 3), loss=torch.zeros(1, dtype=torch.float64, device="cuda"),
             gs=z(L), gsh=z(L, 3, K), sig=z(L), touched=torch.zeros(L, dtype=torch.uint8, device="cuda"))
    dot.dot_render_forward(tree, rays, opts_sig, a["rgb"], None, a["sig"])
    dot.dot.dot_mse_grad(a["rgb"], tgt, a["g"], a["loss"])
    dot.dot_render_backward(tree, rays, plain, a["g"], a["rgb"], a["gs"], a["gsh"], touched=a["touched"])
    b = dict(rgb=z(R, 3), g=z(R, 3), loss=torch.zeros(1, dtype=torch.float64, device="cuda"),
             gs=z(L), gsh=z(L, 3, K), sig=z(L), touched=torch.zeros(L, dtype=torch.uint8, device="cuda"))
    dot.dot.dot_render_forward_backward_mse(tree, rays, opts_sig, tgt, b["rgb"], b["g"], b["gs"],
                                            b["gsh"], b["loss"], b["sig"], b["touched"])
    torch.cuda.synchronize()
    return a, b


def _assert_same_pass(a, b):
    assert torch.equal(a["rgb"], b["rgb"])
    assert torch.equal(a["g"], b["g"])
    assert torch.equal(a["touched"], b["touched"])
    assert float(b["loss"]) == pytest.approx(float(a["loss"]), rel=1e-6)
    for k in ("gs", "gsh", "sig"):
        x, y = a[k].cpu().numpy().astype(np.float64), b[k].cpu().numpy().astype(np.float64)
        assert np.abs(x - y).max() <= 1e-5 * max(np.abs(x).max(), 1e-30), k


@pytest.mark.parametrize("storage,deg", [(si.STORAGE_F32, 2), (si.STORAGE_F16, 3), (si.STORAGE_BF16, 1)])
def test_fused_training_pass_equals_separate_calls(storage, deg):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(45 + deg, max_depth=5, sh_degree=deg, storage=storage, n_prims=4)
    tree = dot.octree_from_scene(scene)
    L, K = tree.n_leaves, (deg + 1) ** 2
    o, d = si.random_rays(5000, 77)
    R = o.shape[0]
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    tgt = torch.from_numpy(np.random.default_rng(2).random((R, 3)).astype(np.float32)).cuda()
    opts = dot.render_opts(background=(0.3, 0.3, 0.9), eps_T=1e-4,
                           signal_mode=dot.dot.DOT_SIGNAL_SUM_ALPHA)
    a, b = _separate_and_fused(dot, tree, rays, opts, tgt, R, L, K)
    assert a["touched"].any()
    _assert_same_pass(a, b)
    tree.free()


def test_fused_training_pass_overflow_rays_march_again():
    """A dense box filling the root at depth 6 without early termination: rays cross up to ~190
    occupied cells, beyond the 32-segment record, and take the backward re-march."""
    import paper_2307_15333_gb300 as dot
    scene = si.box_scene((-1, -1, -1), (1, 1, 1), max_depth=6, sh_degree=1,
                         storage=si.STORAGE_F32, density=(0.01, 0.05), sh_std=0.3)
    tree = dot.octree_from_scene(scene)
    L, K = tree.n_leaves, 4
    o, d = si.random_rays(3000, 78)
    R = o.shape[0]
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    st = dot.dot_render_stats(tree, rays, dot.render_opts(eps_T=0.0))
    assert st["occupied"] > 40 * st["rays_hit"]
    tgt = torch.from_numpy(np.random.default_rng(3).random((R, 3)).astype(np.float32)).cuda()
    opts = dot.render_opts(background=(1, 1, 1), eps_T=0.0, signal_mode=dot.dot.DOT_SIGNAL_MAX_WEIGHT)
    a, b = _separate_and_fused(dot, tree, rays, opts, tgt, R, L, K)
    _assert_same_pass(a, b)
    tree.free()


def test_full_size_fused_training_pass_matches_oracle():
    """The bench's training configuration at full size: a 2^16-ray batch from the 100 views of the
    NeRF-synthetic-shaped scene (2.9 M leaves, FP16, SH degree 3) through the fused pass, against
    the oracle's render, MSE gradient and backward of the same rays.  The fused pass takes dL/dC
    at its own colours; that dL/dC is checked against the oracle's (within the pixel tolerance
    times 2 / 3R) and then handed to the oracle's backward, so the gradients are held to the
    16-bit rule of every other backward test: 2e-3 of the summed magnitudes, plus a floor of
    1e-5 in units of the largest |dL/dC| -- with the grazing-ray budget of a large fast-mode
    batch: at most 0.1% of the leaves with a gradient may exceed it (sliver segments of rays
    that graze a face), none by more than 1e-3 of the largest |dL/dC|."""
    import paper_2307_15333_gb300 as dot
    scene, cams = si.config_nerf_synthetic(100)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    o, d = si.ray_batch(cams, 1 << 16, seed=8123)
    _, _, _, margin = oracle.render(t, lo, size, s64, h64, 3, o, d, eps_T=1e-4, margin=True)
    keep = margin > 1e-3
    assert keep.mean() > 0.99
    o, d = np.ascontiguousarray(o[keep]), np.ascontiguousarray(d[keep])
    R = o.shape[0]
    ref, _, _ = oracle.render(t, lo, size, s64, h64, 3, o, d, eps_T=1e-4)
    tgt = np.where(ref > 0.5, ref - 0.45, ref + 0.45).astype(np.float32)
    rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    L, K = tree.n_leaves, 16
    rgb, g = torch.empty(R, 3, device="cuda"), torch.empty(R, 3, device="cuda")
    gs, gsh = torch.zeros(L, device="cuda"), torch.zeros(L, 3, K, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dot.dot.dot_render_forward_backward_mse(tree, rays, dot.render_opts(eps_T=1e-4),
                                            torch.from_numpy(tgt).cuda(), rgb, g, gs, gsh, loss)
    torch.cuda.synchronize()
    assert np.abs(rgb.cpu().numpy() - ref).max() <= 2e-3
    ref_loss, ref_g = oracle.mse(ref, tgt)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-2)
    g_gpu = g.cpu().numpy().astype(np.float64)
    assert np.abs(g_gpu - ref_g).max() <= 2 * 2e-3 / (3 * R) * 1.001
    rs, rsh, asg, ash = oracle.backward(t, lo, size, s64, h64, 3, o, d, g_gpu, eps_T=1e-4)
    floor = 1e-5 * np.abs(g_gpu).max()
    assert np.abs(rs).max() > 100 * floor
    nb_s, nl_s, w_s = assert_sums_close_grazing(gs.cpu().numpy(), rs, asg, 2e-3, "dsigma", floor)
    nb_h, nl_h, w_h = assert_sums_close_grazing(gsh.cpu().numpy(), rsh, ash, 2e-3, "dsh", floor)
    print(f"grazing exceptions: dsigma {nb_s}/{nl_s} (worst excess {w_s:.3g} x floor), "
          f"dsh {nb_h}/{nl_h} (worst excess {w_h:.3g} x floor)")
    tree.free()
