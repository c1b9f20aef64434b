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

# (prune mode, prune value, sample mode, sample value): rank fractions with many ties, thresholds,
# quantiles
CASES = [(2, 0.2, 2, 0.05), (2, 0.5, 2, 0.01), (1, 0.3, 2, 0.1), (2, 0.07, 1, 2.0), (3, 0.2, 3, 0.05)]


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


# the device's current memory pool (the one cudaMallocAsync draws from), read through the driver
_RESERVED_CURRENT, _RESERVED_HIGH, _USED_CURRENT, _USED_HIGH = 5, 6, 7, 8   # CUmemPool_attribute


class _Pool:
    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_highs(self):
        for attr in (_RESERVED_HIGH, _USED_HIGH):
            zero = ctypes.c_uint64(0)
            assert self.cu.cuMemPoolSetAttribute(self.pool, attr, ctypes.byref(zero)) == 0


def test_noalloc_select_takes_nothing_from_the_memory_pool():
    """The defining property: the call takes no memory from the device's pool (the high-water
    marks of used and reserved pool memory stay at what was in use before it), nor from torch's
    caching allocator, while dot_select_masks on the same input raises the pool's mark."""
    import paper_2307_15333_gb300 as dot
    lib = dot.lib()
    scene = si.box_scene((-2, -2, -2), (2, 2, 2), max_depth=5, sh_degree=0)
    tree = dot.octree_from_scene(scene)
    L = tree.n_leaves
    sig = torch.from_numpy(si.random_signal(L, 77)).cuda()
    opts = dot.select_opts(2, 0.2, 2, 0.05)
    pm = torch.empty(L, dtype=torch.uint8, device="cuda")
    sm = torch.empty(L, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    pool = _Pool()
    for _ in range(2):
        used0, reserved0 = pool.get(_USED_CURRENT), pool.get(_RESERVED_CURRENT)
        torch_allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        pool.reset_highs()
        _call(lib, tree, sig, opts, pm, sm, "dot_select_masks_noalloc")
        torch.cuda.synchronize()
        assert pool.get(_USED_HIGH) <= used0
        assert pool.get(_RESERVED_HIGH) <= reserved0
        assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == torch_allocs0
    # control: the allocating call on the same input does show up in the pool's mark
    used0 = pool.get(_USED_CURRENT)
    pool.reset_highs()
    ref_p = torch.empty_like(pm)
    ref_s = torch.empty_like(sm)
    _call(lib, tree, sig, opts, ref_p, ref_s, "dot_select_masks")
    torch.cuda.synchronize()
    assert pool.get(_USED_HIGH) > used0
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
