"""Serving loop on the GPU over the served tree set (FP32 SH-1 and FP16 SH-3 trees together):
every request's image is the same alone, in a mixed batch, and from a plain dot_render_forward
launch; sampled pixels of every request of a mixed table match the oracle; both servers complete
a real-time trace."""
import numpy as np
import pytest
import torch

import oracle
import seeded_inputs as si
from helpers import assert_pixels_close, oracle_side

pytestmark = pytest.mark.gpu


def _refine_with_oracle_marks(dot, tree, scene):
    """The post-refine training tree: marks from the oracle's max-weight signal of two seeded
    batches of the training views (prune at the 80% quantile, sample the top 5%), applied on the
    GPU and by the oracle; returns the oracle's side (tree, sigma, sh)."""
    t, _, _, s64, h64 = oracle_side(scene)
    lo, size = oracle.root_of(scene)
    _, cams = si.config_train()
    S = np.zeros(s64.shape[0])
    for b in range(2):
        o, d = si.ray_batch(cams, 4096, seed=700 + b)
        oracle.render(t, lo, size, s64, h64, scene.sh_degree, o, d, eps_T=1e-4, signal=S,
                      signal_mode=oracle.SIGNAL_MAX_WEIGHT)
    pm, sm = oracle.select(S.astype(np.float32), oracle.SELECT_QUANTILE, 0.8,
                           oracle.SELECT_FRACTION, 0.05)
    cap = scene.max_depth + 2
    nt, _, so, sho, cnt = oracle.refine(t, s64, h64, pm, sm, cap)
    assert cnt["n_pruned_groups"] > 0 and cnt["n_sampled"] > 0
    pm_t, sm_t = torch.from_numpy(pm).cuda(), torch.from_numpy(sm).cuda()
    plan = dot.dot_refine_plan(tree, pm_t, sm_t, cap)
    lm = torch.empty(plan["n_leaves"], dtype=torch.int32, device="cuda")
    dot.dot_refine_prune(tree, pm_t, sm_t, cap, lm)
    torch.cuda.synchronize()
    return nt, so, sho


@pytest.fixture(scope="module")
def served():
    import paper_2307_15333_gb300 as dot
    scenes, refined, poses = si.config_serving()
    trees = [dot.octree_from_scene(s) for s in scenes]
    sides = []
    for sc, tr, ref in zip(scenes, trees, refined):
        if ref:
            sides.append(_refine_with_oracle_marks(dot, tr, sc))
        else:
            t, _, _, s64, h64 = oracle_side(sc)
            sides.append((t, s64, h64))
    yield scenes, trees, sides, poses
    for t in trees:
        t.free()


def _requests(poses, n, seed):
    from paper_2307_15333_gb300 import serve
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        w, h = si.SERVE_RESOLUTIONS[i % 5]
        reqs.append(serve.Request(i, i % 4, w, h, poses(rng, i % 4, w, h), 0.0))
    return reqs


def test_served_trees_mix_storage_and_degree(served):
    from paper_2307_15333_gb300 import serve
    scenes, trees, _, _ = served
    assert {(t.storage, t.sh_degree) for t in trees} == {(si.STORAGE_F32, 1), (si.STORAGE_F16, 3)}
    assert serve.slot_groups(trees) == [[0, 1], [2, 3]]
    assert trees[1].n_leaves != trees[0].n_leaves


def test_alone_equals_mixed_equals_plain(served):
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    _, trees, _, poses = served
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    reqs = _requests(poses, 10, 0)
    srv = serve.BatchedServer(trees, opts, pool_floats=64 << 20, max_slots=16)
    mixed, alone = srv.render_alone_and_mixed(reqs)
    for r, m, a in zip(reqs, mixed, alone):
        assert torch.equal(m, a), f"request {r.rid} differs alone vs mixed"
        cam = torch.from_numpy(r.camera).cuda().view(1, 18)
        ref = torch.empty(r.width * r.height, 3, device="cuda")
        dot.dot_render_forward(trees[r.tree], dot.rays_cameras(cam, r.width, r.height), opts, ref)
        torch.cuda.synchronize()
        assert torch.equal(m.view(-1, 3), ref), f"request {r.rid} differs from dot_render_forward"
        assert float(m.std()) > 0.01
    assert all(t.status() == 0 for t in trees)


def test_slots_match_oracle(served):
    """One mixed slot table (10 requests over the 5 resolutions and the 4 trees: two storage
    types and SH degrees) rendered by one graph replay; 500 seeded pixels of every request
    against the oracle's render of the same camera rays, at the tolerance of the tree's storage
    (FP32 exact mode: 1e-5 relative; FP16: 2e-3 absolute)."""
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    scenes, trees, sides, poses = served
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    reqs = _requests(poses, 10, 11)
    srv = serve.BatchedServer(trees, opts, pool_floats=64 << 20, max_slots=16)
    for r in reqs:
        r.offset = srv.pool.alloc(r.floats)
    srv.submit(reqs, srv.tables[0])
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for r in reqs:
        img = srv.pool_t[r.offset: r.offset + r.floats].view(-1, 3).cpu().numpy()
        cam = si.Camera.unpack(r.camera)
        pix = rng.choice(r.width * r.height, 500, replace=False)
        o, d = si.camera_rays(cam, pix)
        sc = scenes[r.tree]
        t, s64, h64 = sides[r.tree]
        lo, size = oracle.root_of(sc)
        ref, _, _ = oracle.render(t, lo, size, s64, h64, sc.sh_degree, o, d, bg=(1, 1, 1),
                                  eps_T=1e-4)
        assert_pixels_close(img[pix], ref, sc.storage, what=f"request {r.rid} (tree {r.tree})")
    assert all(t.status() == 0 for t in trees)


def test_servers_complete_a_trace(served):
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    _, trees, _, poses = served
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    for cls in (serve.BatchedServer, serve.PlainServer):
        trace = serve.poisson_trace(150, 300.0, 4, si.SERVE_RESOLUTIONS, poses, seed=5)
        srv = cls(trees, opts, pool_floats=256 << 20)
        srv.run(trace)
        assert all(r.done >= r.arrival for r in trace)
        st = serve.percentiles(trace)
        assert 0 < st["p50_ms"] <= st["p99_ms"] < 1000
