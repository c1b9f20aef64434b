"""dot_select_masks_noalloc: the selection for callers that cannot have the library allocate
device memory (a process that reserves its whole memory budget up front, or whose allocation path
may block or fail under memory pressure).  It must give exactly the marks of dot_select_masks,
call after call, although every call reuses one fixed array in the library's device memory.

This file is collected last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import seeded_inputs as si

pytestmark = pytest.mark.gpu

# (prune mode, prune value, sample mode, sample value): rank fractions with many ties, thresholds
CASES = [(2, 0.2, 2, 0.05), (2, 0.5, 2, 0.01), (1, 0.3, 2, 0.1), (2, 0.07, 1, 2.0)]


def _call(lib, tree, sig, opts, pm, sm, name):
    fn = getattr(lib, name)
    rc = fn(tree.handle, ctypes.c_void_p(sig.data_ptr()), ctypes.byref(opts),
            ctypes.c_void_p(pm.data_ptr()), ctypes.c_void_p(sm.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.dot_last_error().decode()


@pytest.mark.parametrize("depth", [2, 5, 7])
def test_noalloc_select_matches_allocating_select_twice(depth):
    import paper_2307_15333_gb300 as dot
    lib = dot.lib()
    scene = si.box_scene((-2, -2, -2), (2, 2, 2), max_depth=depth, sh_degree=0)
    tree = dot.octree_from_scene(scene)                     # 8^depth leaves
    L = tree.n_leaves
    for call, (pmode, pval, smode, sval) in enumerate(CASES[:2] if depth == 2 else CASES):
        sig = torch.from_numpy(si.random_signal(L, 100 * depth + call)).cuda()
        opts = dot.select_opts(pmode, pval, smode, sval)
        ref_p = torch.empty(L, dtype=torch.uint8, device="cuda")
        ref_s = torch.empty(L, dtype=torch.uint8, device="cuda")
        _call(lib, tree, sig, opts, ref_p, ref_s, "dot_select_masks")
        # two calls in a row on the shared scratch; the masks start as garbage each time
        for _ in range(2):
            pm = torch.full((L,), 7, dtype=torch.uint8, device="cuda")
            sm = torch.full((L,), 7, dtype=torch.uint8, device="cuda")
            _call(lib, tree, sig, opts, pm, sm, "dot_select_masks_noalloc")
            torch.cuda.synchronize()
            assert torch.equal(pm, ref_p) and torch.equal(sm, ref_s)
    tree.free()


def test_noalloc_select_on_the_refine_workload():
    """The config-scale selection (2.9 M leaves, bottom 20% / top 5%), twice in a row."""
    import paper_2307_15333_gb300 as dot
    lib = dot.lib()
    scene = si.nerf_synthetic_scene()
    tree = dot.octree_from_scene(scene)
    L = tree.n_leaves
    sig = torch.from_numpy(si.random_signal(L, 9)).cuda()
    opts = dot.select_opts(2, 0.2, 2, 0.05)
    ref_p = torch.empty(L, dtype=torch.uint8, device="cuda")
    ref_s = torch.empty(L, dtype=torch.uint8, device="cuda")
    _call(lib, tree, sig, opts, ref_p, ref_s, "dot_select_masks")
    for _ in range(2):
        pm = torch.empty(L, dtype=torch.uint8, device="cuda")
        sm = torch.empty(L, dtype=torch.uint8, device="cuda")
        _call(lib, tree, sig, opts, pm, sm, "dot_select_masks_noalloc")
        torch.cuda.synchronize()
        assert torch.equal(pm, ref_p) and torch.equal(sm, ref_s)
        assert int(sm.sum()) == int(np.ceil(0.05 * L))
    tree.free()
