"""The C-ABI library loads and exports every entry point include/dot.h declares (no GPU needed),
and host-side argument checks answer without touching a device."""
import ctypes
import os
import re


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dot_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dot_octree_build", "dot_render_forward", "dot_render_backward",
                     "dot_accumulate_signal", "dot_refine_prune", "dot_select_masks"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2307_15333_gb300 import dot
    L = dot.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(dot.ENTRY_POINTS) == set(_declared())
    assert dot.dot_version() == 100


def test_host_side_argument_errors():
    from paper_2307_15333_gb300 import dot
    L = dot.lib()
    h = ctypes.c_void_p()
    assert L.dot_octree_build(None, None, None, ctypes.byref(h)) == dot.DOT_ERR_INVALID_ARG
    assert b"NULL" in L.dot_last_error()
    import numpy as np
    d = dot.build_desc((0, 0, 0), 1.0, 0, 1, 0, np.zeros((0, 8), np.int64))
    assert L.dot_octree_build(ctypes.byref(d), None, None, ctypes.byref(h)) == dot.DOT_ERR_INVALID_ARG
    d = dot.build_desc((0, 0, 0), 1.0, 3, 4, 0, np.zeros((0, 8), np.int64))
    assert L.dot_octree_build(ctypes.byref(d), None, None, ctypes.byref(h)) == dot.DOT_ERR_UNSUPPORTED
    bad = np.array([[7, 0, 0, 0, 0, 0, 0, 0]], np.int64)
    d = dot.build_desc((0, 0, 0), 1.0, 3, 1, 0, bad)
    assert L.dot_octree_build(ctypes.byref(d), None, None, ctypes.byref(h)) == dot.DOT_ERR_INVALID_ARG
    assert L.dot_tree_get_info(None, None) == dot.DOT_ERR_INVALID_ARG
    assert L.dot_tree_import(None, None, None, ctypes.byref(h)) == dot.DOT_ERR_INVALID_ARG


def test_import_rejects_malformed_trees_on_host():
    """dot_tree_import validates structure before touching the device."""
    import numpy as np
    from paper_2307_15333_gb300 import dot
    L = dot.lib()
    child = np.array([[-1, -2, -3, -4, -5, -6, -7, -9]], np.int32)     # leaf 8 does not exist
    host = dot.dot_host_tree()
    arrs = dict(child=child, node_parent=np.array([-1], np.int32), node_key=np.array([1], np.uint64),
                leaf_parent=np.zeros(8, np.int32), leaf_key=np.arange(8, 16, dtype=np.uint64),
                sigma=np.zeros(8, np.float32), sh=np.zeros((8, 3, 1), np.float32))
    host.n_nodes, host.n_leaves, host.sh_degree, host.storage, host.half_size = 1, 8, 0, 0, 1.0
    for k, v in arrs.items():
        setattr(host, k, v.ctypes.data_as(ctypes.c_void_p))
    h = ctypes.c_void_p()
    assert L.dot_tree_import(ctypes.byref(host), None, None, ctypes.byref(h)) == dot.DOT_ERR_INVALID_ARG
    assert b"leaf" in L.dot_last_error()


def test_render_views_host_workspace_sizes():
    """Workspace of dot_render_views_host: the cameras (72 B each), the view order (4 B each), then
    up to three chunk buffers of a full chunk (about 2^23 rays) each, every part rounded up to
    256 bytes; worked by hand."""
    from paper_2307_15333_gb300 import dot
    f = dot.dot_render_views_host_workspace
    # 100 views of 800x800 (64 M rays): chunks of 13 views (7 full, then 5, 2, 1, 1), three buffers
    # of 13 x 640000 x 12 B
    assert f(100, 800, 800) == 7424 + 512 + 3 * 99840000
    assert f(100, 800, 800, True) == 7424 + 512 + 3 * (99840000 + 33280000)
    # 7 views of 320x240 (537600 rays): one chunk, one buffer
    assert f(7, 320, 240) == 512 + 256 + 6451200
    assert f(7, 320, 240, True) == 512 + 256 + 6451200 + 2150400
    # one 8x8 view: 768 B of colour
    assert f(1, 8, 8) == 256 + 256 + 768
    # two 4096x4096 views (2 x 2^24 rays): one view per chunk, two buffers
    assert f(2, 4096, 4096) == 256 + 256 + 2 * 201326592
    assert f(0, 800, 800) == 0
    for bad in ((-1, 8, 8), (65536, 8, 8), (1, 0, 8), (1, 8, 65537)):
        assert f(*bad, 0) == -1


def test_probe_argument_errors():
    """The L2 read-bandwidth probe checks its buffer, size and pass count on the host."""
    import ctypes as C
    from paper_2307_15333_gb300 import dot
    L = dot.lib()
    assert L.dot_probe_l2_read(None, 1024, 1, None, None) == dot.DOT_ERR_INVALID_ARG
    buf = C.create_string_buffer(64)
    aligned = (C.addressof(buf) + 15) & ~15
    assert L.dot_probe_l2_read(C.c_void_p(aligned), 24, 1, None, None) == dot.DOT_ERR_INVALID_ARG
    assert L.dot_probe_l2_read(C.c_void_p(aligned + 4), 16, 1, None, None) == dot.DOT_ERR_INVALID_ARG
    assert L.dot_probe_l2_read(C.c_void_p(aligned), 16, 0, None, None) == dot.DOT_ERR_INVALID_ARG
