"""The training step on the GPU (MSE gradient, RMSProp fused with zeroing the gradients) and the
Algorithm 1 loop (optimisation steps, then recursive pruning and sampling) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import assert_pixels_close, assert_sums_close, oracle_side

pytestmark = pytest.mark.gpu


def _ulp(x, storage):
    """Spacing of the storage format at |x|."""
    x = np.abs(np.asarray(x, np.float64))
    if storage == si.STORAGE_F32:
        return np.spacing(x.astype(np.float32)).astype(np.float64)
    if storage == si.STORAGE_F16:
        return np.spacing(x.astype(np.float16)).astype(np.float64)
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 2.0 ** (e - 7)


@pytest.mark.parametrize("R", [0, 1, 37, 4099, 70001])
def test_mse_grad_matches_oracle(R):
    import paper_2307_15333_gb300 as dot
    rng = np.random.default_rng(R)
    rgb = rng.random((R, 3)).astype(np.float32)
    tgt = rng.random((R, 3)).astype(np.float32)
    g = torch.full((R, 3), 7.0, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    dot.dot.dot_mse_grad(torch.from_numpy(rgb).cuda(), torch.from_numpy(tgt).cuda(), g, loss)
    torch.cuda.synchronize()
    if R == 0:
        assert float(loss) == 0.0
        return
    ref_loss, ref_g = oracle.mse(rgb, tgt)
    np.testing.assert_allclose(g.cpu().numpy(), ref_g, rtol=1e-6, atol=1e-12)
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)


@pytest.mark.parametrize("storage,deg", [(st, d) for st in (si.STORAGE_F32, si.STORAGE_F16, si.STORAGE_BF16)
                                         for d in range(4)])
def test_rmsprop_matches_oracle(storage, deg):
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(60 + deg, max_depth=4, sh_degree=deg, storage=storage, n_prims=3)
    tree = dot.octree_from_scene(scene)
    L, K = tree.n_leaves, (deg + 1) ** 2
    rng = np.random.default_rng(deg + 10 * storage)
    gs = (rng.normal(size=L) * 0.1).astype(np.float32)
    gsh = (rng.normal(size=(L, 3, K)) * 0.01).astype(np.float32)
    gs[::7] = 0.0
    ms_s = (rng.random(L) * 0.01).astype(np.float32)
    ms_sh = (rng.random((L, 3, K)) * 1e-4).astype(np.float32)
    ms_sh[::5] = 0.0
    p_s = tree.sigma.float().cpu().numpy().astype(np.float64)
    p_sh = tree.sh.float().cpu().numpy().astype(np.float64)
    t_gs, t_gsh = torch.from_numpy(gs).cuda(), torch.from_numpy(gsh).cuda()
    t_ms, t_msh = torch.from_numpy(ms_s).cuda(), torch.from_numpy(ms_sh).cuda()
    opts = dot.dot.rmsprop_opts(lr_sigma=0.1, lr_sh=0.01, rho=0.9, eps=1e-8)
    dot.dot.dot_rmsprop_step(tree, t_gs, t_gsh, t_ms, t_msh, opts)
    torch.cuda.synchronize()
    assert not t_gs.any() and not t_gsh.any()
    for p0, g, m0, lr, got_p, got_m in ((p_s, gs, ms_s, 0.1, tree.sigma, t_ms),
                                        (p_sh, gsh, ms_sh, 0.01, tree.sh, t_msh)):
        ref_p, ref_m = oracle.rmsprop(p0, m0, g, lr, 0.9, 1e-8)
        got_m = got_m.cpu().numpy().astype(np.float64)
        np.testing.assert_allclose(got_m, ref_m, rtol=1e-6, atol=1e-30)
        got_p = got_p.float().cpu().numpy().astype(np.float64)
        upd = np.abs(ref_p - p0)
        lim = 1e-6 * (np.abs(p0) + upd)
        if storage != si.STORAGE_F32:
            lim = lim + _ulp(ref_p, storage)
        d = np.abs(got_p - ref_p)
        assert (d <= lim).all(), f"{(d > lim).sum()} parameters beyond tolerance, worst {d.max():.3g}"
    tree.free()


def _oracle_remap(t, lm, a, merge):
    return oracle.remap_leaf_values(t, lm, a, merge)


def test_training_loop_matches_oracle():
    """Three optimisation steps (forward with the fused SUM_ALPHA signal, MSE gradient, backward,
    RMSProp) on an FP32 scene, then Algorithm 1's recursive pruning and top-gamma sampling, all on
    the GPU through the Trainer, against the same sequence composed from the oracle."""
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.train import Trainer
    scene = si.random_scene(70, max_depth=5, sh_degree=1, storage=si.STORAGE_F32, n_prims=3)
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    bg = (1.0, 1.0, 1.0)
    opts = dot.render_opts(background=bg, eps_T=0.0)
    lr_s, lr_h, rho, eps = 0.1, 0.01, 0.9, 1e-3
    tr = Trainer(tree, opts, dot.dot.rmsprop_opts(lr_s, lr_h, rho, eps),
                 signal_mode=dot.dot.DOT_SIGNAL_SUM_ALPHA)
    ms_s, ms_h = np.zeros_like(s64), np.zeros_like(h64)
    S = np.zeros(s64.shape[0])
    Sabs = np.zeros(s64.shape[0])
    rng = np.random.default_rng(1)
    for b in range(3):
        o, d = si.random_rays(3000, 300 + b)
        tgt = rng.random((3000, 3)).astype(np.float32)
        rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
        tr.step(rays, torch.from_numpy(tgt).cuda())
        # oracle: the same step, parameters rounded to the FP32 storage after the update
        rgb, _, _ = oracle.render(t, lo, size, s64, h64, 1, o, d, bg=bg, eps_T=0.0, signal=S,
                                  signal_mode=oracle.SIGNAL_SUM_ALPHA)
        _, g = oracle.mse(rgb, tgt)
        gs, gsh, _, _ = oracle.backward(t, lo, size, s64, h64, 1, o, d, g, bg=bg, eps_T=0.0)
        s64, ms_s = oracle.rmsprop(s64, ms_s, gs, lr_s, rho, eps)
        h64, ms_h = oracle.rmsprop(h64, ms_h, gsh, lr_h, rho, eps)
        s64 = s64.astype(np.float32).astype(np.float64)
        h64 = h64.astype(np.float32).astype(np.float64)
    tr.flush()
    torch.cuda.synchronize()
    assert tree.status() == 0
    got_s = tree.sigma.cpu().numpy().astype(np.float64)
    got_h = tree.sh.cpu().numpy().astype(np.float64)
    # an FP32 gradient error dg moves an update by at most lr dg / eps (|g| << eps) and not at all
    # once |g| >> eps; the FP32 gradients match to ~1e-5 of their summed magnitudes
    np.testing.assert_allclose(got_s, s64, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(got_h, h64, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(tr.ms_sigma.cpu().numpy(), ms_s, rtol=1e-3, atol=1e-9)
    sig = tr.signal.cpu().numpy().astype(np.float64)
    assert_sums_close(sig, S, S, 1e-5, "signal")

    # Algorithm 1 pruning (recursive) and sampling on the accumulated signal: tau and gamma are
    # placed in gaps of the oracle's signal so that FP32 sums cannot flip a decision
    pos = np.sort(S[S > 0])
    assert pos.size > 20
    gaps = [(pos[i + 1] - pos[i]) / pos[i + 1] for i in range(pos.size // 4, pos.size // 2)]
    i = pos.size // 4 + int(np.argmax(gaps))
    tau = 0.5 * (pos[i] + pos[i + 1])
    nt, so, sho, S2, (ms_s2, ms_h2), passes = oracle.prune_recursive(
        t, s64, h64, S.astype(np.float32), tau, d_cap=7, aux=(ms_s, ms_h))
    L2 = nt["leaf_key"].size
    order = np.lexsort((np.arange(L2), -S2))
    k = max(1, int(np.ceil(0.05 * L2)))
    while k < L2 and abs(S2[order[k - 1]] - S2[order[k]]) <= 1e-4 * abs(S2[order[k - 1]]):
        k += 1
    gamma = (k - 0.5) / L2
    pm2, smk = oracle.select(S2.astype(np.float32), oracle.SELECT_NONE, 0.0,
                             oracle.SELECT_FRACTION, gamma)
    nt3, lm3, so3, sho3, cnt3 = oracle.refine(nt, so, sho, pm2, smk, 7)
    res = tr.refine(tau, gamma, depth_cap=7, recursive=True)
    assert [p["n_pruned_groups"] for p in res["passes"][:-1]] == [p["n_pruned_groups"] for p in passes]
    ex = tree.export()
    for key in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        assert np.array_equal(ex[key], nt3[key]), key
    np.testing.assert_array_equal(tr.leaf_map.cpu().numpy(), lm3)
    np.testing.assert_allclose(ex["sigma"].astype(np.float64), so3, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(ex["sh"].astype(np.float64), sho3, rtol=1e-5, atol=1e-4)
    ms3 = oracle.remap_leaf_values(nt, lm3, ms_s2, "mean")
    np.testing.assert_allclose(tr.ms_sigma.cpu().numpy(), ms3, rtol=1e-3, atol=1e-9)
    assert tr.L == nt3["leaf_key"].size and tr.grad_sigma.shape[0] == tr.L
    tree.free()


@pytest.mark.parametrize("storage", [si.STORAGE_F32, si.STORAGE_F16, si.STORAGE_BF16])
def test_sparse_rmsprop_equals_dense(storage):
    """Six steps in which a random fifth of the leaves have gradients: the sparse update (touched
    leaves only, deferred decay, final flush) against the oracle's dense RMSProp of every leaf."""
    import paper_2307_15333_gb300 as dot
    scene = si.random_scene(61, max_depth=5, sh_degree=3, storage=storage, n_prims=3)
    tree = dot.octree_from_scene(scene)
    L, K = tree.n_leaves, 16
    rng = np.random.default_rng(storage)
    p_s = tree.sigma.float().cpu().numpy().astype(np.float64)
    p_h = tree.sh.float().cpu().numpy().astype(np.float64)
    ms_s, ms_h = np.zeros(L), np.zeros((L, 3, K))
    t_gs = torch.zeros(L, device="cuda")
    t_gsh = torch.zeros(L, 3, K, device="cuda")
    t_ms, t_msh = torch.zeros(L, device="cuda"), torch.zeros(L, 3, K, device="cuda")
    touched = torch.zeros(L, dtype=torch.uint8, device="cuda")
    last = torch.zeros(L, dtype=torch.int32, device="cuda")
    work = torch.empty(L + 1, dtype=torch.int32, device="cuda")
    opts = dot.dot.rmsprop_opts(lr_sigma=0.1, lr_sh=0.01, rho=0.9, eps=1e-8)
    moved_s, moved_h = np.zeros(L), np.zeros((L, 3, K))     # sum of |update| per entry
    for step in range(1, 7):
        hit = rng.random(L) < 0.2
        gs = np.where(hit, rng.normal(size=L) * 0.1, 0.0).astype(np.float32)
        gsh = np.where(hit[:, None, None], rng.normal(size=(L, 3, K)) * 0.01, 0.0).astype(np.float32)
        t_gs.copy_(torch.from_numpy(gs))
        t_gsh.copy_(torch.from_numpy(gsh))
        touched.copy_(torch.from_numpy(hit.astype(np.uint8)))
        dot.dot.dot_rmsprop_step_sparse(tree, t_gs, t_gsh, t_ms, t_msh, touched, last, step, work, opts)
        q_s, ms_s = oracle.rmsprop(p_s, ms_s, gs, 0.1, 0.9, 1e-8)
        q_h, ms_h = oracle.rmsprop(p_h, ms_h, gsh, 0.01, 0.9, 1e-8)
        moved_s += np.abs(q_s - p_s)
        moved_h += np.abs(q_h - p_h)
        p_s, p_h = q_s, q_h
        # the stored parameters are what the next step reads
        p_s = si.storage_to_f64(si.round_to_storage(p_s.astype(np.float32), storage), storage)
        p_h = si.storage_to_f64(si.round_to_storage(p_h.astype(np.float32), storage), storage)
        torch.cuda.synchronize()
        assert not touched.any() and not t_gs.any() and not t_gsh.any()
    dot.dot.dot_rmsprop_flush(tree, t_ms, t_msh, last, 6, opts)
    torch.cuda.synchronize()
    assert (last.cpu().numpy() == 6).all()
    np.testing.assert_allclose(t_ms.cpu().numpy(), ms_s, rtol=1e-5, atol=1e-30)
    np.testing.assert_allclose(t_msh.cpu().numpy(), ms_h, rtol=1e-5, atol=1e-30)
    # each step rounds to the storage type (one ulp either way near a rounding boundary) after an
    # FP32 update whose error is ~1e-6 of the magnitudes involved
    for got, ref, moved in ((tree.sigma, p_s, moved_s), (tree.sh, p_h, moved_h)):
        got = got.float().cpu().numpy().astype(np.float64)
        lim = _ulp(ref, storage) + 1e-6 * (np.abs(ref) + moved)
        d = np.abs(got - ref)
        assert (d <= lim).mean() > 0.999 and (d <= 3 * lim).all(), f"worst {(d / lim).max():.3g} x limit"
    tree.free()


def test_fit_runs_algorithm_1():
    """Trainer.fit: epochs of optimisation over the caller's batches with the signal accumulated,
    pruning and sampling every T epochs (Algorithm 1).  Trained toward the renders of a tree of the
    same structure with other seeded parameters, the epoch MSE falls; each refine reports its
    plan and changes the leaves; every step's render stays in step with the oracle's render of
    the trained parameters."""
    import dataclasses
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.train import Trainer
    scene = si.random_scene(73, max_depth=5, sh_degree=1, storage=si.STORAGE_F32, n_prims=3)
    tree = dot.octree_from_scene(scene)
    goal = dot.octree_from_scene(dataclasses.replace(scene, seed=scene.seed + 17))
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    batches = []
    for b in range(4):
        o, d = si.random_rays(4096, 900 + b)
        rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
        tgt = torch.empty(4096, 3, device="cuda")
        dot.dot_render_forward(goal, rays, opts, tgt)
        batches.append((rays, tgt))
    rng = np.random.default_rng(4)

    def epoch(i):  # the epoch's batches in a permuted order
        return [batches[j] for j in rng.permutation(len(batches))]

    tr = Trainer(tree, opts, dot.dot.rmsprop_opts(0.1, 0.01, 0.9, 1e-8),
                 signal_mode=dot.dot.DOT_SIGNAL_MAX_WEIGHT)
    refines = []
    L0 = tree.n_leaves
    losses = tr.fit(epoch, epochs=6, T=3, tau=1e-3, gamma=0.02, depth_cap=6,
                    on_refine=lambda i, plan: refines.append((i, plan)))
    torch.cuda.synchronize()
    assert tree.status() == 0
    assert [i for i, _ in refines] == [3, 6]
    assert all(p["passes"] for _, p in refines) and tree.n_leaves != L0
    assert losses[2] < losses[1] < losses[0] and losses[-1] < losses[0], losses
    # the trained tree renders as the oracle's render of its exported parameters
    ex = tree.export()
    t = {k: ex[k] for k in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key")}
    lo, size = oracle.root_of(scene)
    o, d = si.random_rays(3000, 77)
    got = torch.empty(3000, 3, device="cuda")
    dot.dot_render_forward(tree, dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()),
                           opts, got)
    s64 = ex["sigma"].astype(np.float64)
    h64 = ex["sh"].astype(np.float64)
    ref, _, _ = oracle.render(t, lo, size, s64, h64, 1, o, d, eps_T=1e-4)
    assert_pixels_close(got.cpu().numpy(), ref, scene.storage)
    tree.free()
    goal.free()


def _fraction_in_gap(S, frac, largest_first):
    """A rank fraction near `frac` whose k-th and (k+1)-th signals in the selection order are both
    exactly zero (equal keys, taken in leaf-id order on both sides) or apart by more than 1e-4 of
    their size, so that FP32 sums cannot move the boundary."""
    L = S.size
    order = np.lexsort((np.arange(L), -S if largest_first else S))
    want = max(1, int(np.ceil(frac * L)))
    best = None
    for k in range(max(1, want // 2), min(L - 1, 2 * want) + 1):
        a, b = S[order[k - 1]], S[order[k]]
        if (a == 0 and b == 0) or abs(a - b) > 1e-4 * max(abs(a), abs(b)):
            if best is None or abs(k - want) < abs(best - want):
                best = k
    assert best is not None
    return (best - 0.5) / L


def _quantile_in_gap(S, frac):
    """A quantile fraction near `frac` whose bound (the k-th smallest signal) is apart from both
    of its neighbours in sorted order by more than 1e-4 of its size, so that FP32 sums cannot
    move a leaf across it."""
    v = np.sort(S)
    want = max(2, int(np.ceil(frac * S.size)))
    best = None
    for k in range(2, S.size):
        a, b, c = v[k - 2], v[k - 1], v[k]
        if b > 0 and b - a > 1e-4 * b and c - b > 1e-4 * c:
            if best is None or abs(k - want) < abs(best - want):
                best = k
    assert best is not None
    return (best - 0.5) / S.size


def test_config3_training_matches_oracle_loop():
    """A short run of the differentiable-training configuration: the tiny FP32 sphere scene,
    targets rendered from the seeded perturbed copy of its parameters, batches of rays from its
    800x800 views, two fused training steps with the MAX_WEIGHT signal, a refine (prune at a
    quantile of the signal, then sample a top fraction of the merged signal), and two more
    steps on the refined tree -- through Trainer on the GPU and composed from the oracle, with the
    same targets.  Structure and leaf map bit-exact; parameters as in the other loop test."""
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300.train import Trainer
    scene, cams = si.config_train()
    tree = dot.octree_from_scene(scene)
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    ex = tree.export()
    sg, shg = si.perturbed_params(ex["sigma"], ex["sh"], seed=2002)
    goal = dot.dot.dot_tree_import(dict(ex, sigma=sg, sh=shg))
    bg = (1.0, 1.0, 1.0)
    opts = dot.render_opts(background=bg, eps_T=0.0)
    batches = []
    for b in range(4):
        o, d = si.ray_batch(cams, 4096, seed=600 + b)
        tgt, _, _ = oracle.render(t, lo, size, sg.astype(np.float64), shg.astype(np.float64), 1,
                                  o, d, bg=bg, eps_T=0.0)
        rays = dot.rays_buffer(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
        # the GPU's render of the perturbed copy is the oracle's (FP32 tolerance)
        gt = torch.empty(4096, 3, device="cuda")
        dot.dot_render_forward(goal, rays, opts, gt)
        torch.cuda.synchronize()
        assert_pixels_close(gt.cpu().numpy(), tgt, si.STORAGE_F32)
        batches.append((o, d, rays, tgt.astype(np.float32)))
    goal.free()
    lr_s, lr_h, rho, eps = 0.1, 0.01, 0.9, 1e-3
    tr = Trainer(tree, opts, dot.dot.rmsprop_opts(lr_s, lr_h, rho, eps),
                 signal_mode=dot.dot.DOT_SIGNAL_MAX_WEIGHT)
    ms_s, ms_h = np.zeros_like(s64), np.zeros_like(h64)
    S = np.zeros(s64.shape[0])

    def oracle_step(t, s64, h64, ms_s, ms_h, S, o, d, tgt):
        rgb, _, _ = oracle.render(t, lo, size, s64, h64, 1, o, d, bg=bg, eps_T=0.0, signal=S,
                                  signal_mode=oracle.SIGNAL_MAX_WEIGHT)
        _, g = oracle.mse(rgb, tgt)
        gs, gsh, _, _ = oracle.backward(t, lo, size, s64, h64, 1, o, d, g, bg=bg, eps_T=0.0)
        s64, ms_s = oracle.rmsprop(s64, ms_s, gs, lr_s, rho, eps)
        h64, ms_h = oracle.rmsprop(h64, ms_h, gsh, lr_h, rho, eps)
        return (s64.astype(np.float32).astype(np.float64),
                h64.astype(np.float32).astype(np.float64), ms_s, ms_h)

    for o, d, rays, tgt in batches[:2]:
        tr.step(rays, torch.from_numpy(tgt).cuda())
        s64, h64, ms_s, ms_h = oracle_step(t, s64, h64, ms_s, ms_h, S, o, d, tgt)
    torch.cuda.synchronize()
    assert_sums_close(tr.signal.cpu().numpy(), S, S, 1e-5, "signal")
    # refine: prune at a quantile of the signal (placed in a gap near 0.8: on this tree every
    # sibling group has a leaf seen by some ray, so lower quantiles merge nothing), then sample
    # the top fraction of the merged signal
    f_p = _quantile_in_gap(S, 0.8)
    pm, _ = oracle.select(S.astype(np.float32), oracle.SELECT_QUANTILE, f_p)
    nt, lm, so, sho, cnt = oracle.refine(t, s64, h64, pm, np.zeros_like(pm), scene.max_depth + 2)
    assert cnt["n_pruned_groups"] > 0
    S2 = oracle.remap_leaf_values(t, lm, S, "max")
    ms_s = oracle.remap_leaf_values(t, lm, ms_s, "mean")
    ms_h = oracle.remap_leaf_values(t, lm, ms_h, "mean")
    f_s = _fraction_in_gap(S2, 0.05, largest_first=True)
    _, sm = oracle.select(S2.astype(np.float32), oracle.SELECT_NONE, 0.0, oracle.SELECT_FRACTION, f_s)
    nt2, lm2, so2, sho2, cnt = oracle.refine(nt, so, sho, np.zeros_like(sm), sm, scene.max_depth + 2)
    assert cnt["n_sampled"] > 0
    ms_s = oracle.remap_leaf_values(nt, lm2, ms_s, "mean")
    ms_h = oracle.remap_leaf_values(nt, lm2, ms_h, "mean")
    res = tr.refine(f_p, f_s, depth_cap=scene.max_depth + 2, recursive=False,
                    prune_mode=dot.dot.DOT_SELECT_QUANTILE, sample_mode=dot.dot.DOT_SELECT_FRACTION)
    assert res["n_leaves"] == nt2["leaf_key"].size
    ex = tree.export()
    for key in ("child", "node_parent", "node_key", "leaf_parent", "leaf_key"):
        assert np.array_equal(ex[key], nt2[key]), key
    np.testing.assert_array_equal(tr.leaf_map.cpu().numpy(), lm2)
    # two more steps on the refined tree
    t, s64, h64 = nt2, so2, sho2
    S = np.zeros(s64.shape[0])
    for o, d, rays, tgt in batches[2:]:
        tr.step(rays, torch.from_numpy(tgt).cuda())
        s64, h64, ms_s, ms_h = oracle_step(t, s64, h64, ms_s, ms_h, S, o, d, tgt)
    tr.flush()
    torch.cuda.synchronize()
    assert tree.status() == 0
    np.testing.assert_allclose(tree.sigma.cpu().numpy().astype(np.float64), s64, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(tree.sh.cpu().numpy().astype(np.float64), h64, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(tr.ms_sigma.cpu().numpy(), ms_s, rtol=1e-3, atol=1e-9)
    tree.free()
