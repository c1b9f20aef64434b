"""Serving loop on the GPU: every request's image is the same alone, in a mixed batch, and from
a plain dot_render_forward launch; both servers complete a real-time trace."""
import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served():
    import paper_2307_15333_gb300 as dot
    scenes, poses = si.config_serving()
    trees = [dot.octree_from_scene(s) for s in scenes]
    yield trees, poses
    for t in trees:
        t.free()


def test_alone_equals_mixed_equals_plain(served):
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    trees, poses = served
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(10):
        w, h = si.SERVE_RESOLUTIONS[i % 5]
        tr = int(rng.integers(0, 4))
        reqs.append(serve.Request(i, tr, w, h, poses(rng, tr, w, h), 0.0))
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


def test_servers_complete_a_trace(served):
    import paper_2307_15333_gb300 as dot
    from paper_2307_15333_gb300 import serve
    trees, poses = served
    opts = dot.render_opts(background=(1, 1, 1), eps_T=1e-4)
    for cls in (serve.BatchedServer, serve.PlainServer):
        trace = serve.poisson_trace(150, 300.0, 4, si.SERVE_RESOLUTIONS, poses, seed=5)
        srv = cls(trees, opts, pool_floats=256 << 20)
        srv.run(trace)
        assert all(r.done >= r.arrival for r in trace)
        st = serve.percentiles(trace)
        assert 0 < st["p50_ms"] <= st["p99_ms"] < 1000
