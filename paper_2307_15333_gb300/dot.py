"""Thin ctypes binding of ``libdot.so`` (include/dot.h), with the same entry-point names.

Only argument marshalling lives here: every step of the path runs in the CUDA library.  Device
buffers are torch CUDA tensors (PyTorch supplies device memory and the current stream).  If the
library cannot be loaded the import fails; there is no fallback.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

# ----------------------------------------------------------------------------------------------
# constants (mirror include/dot.h)
# ----------------------------------------------------------------------------------------------
DOT_OK = 0
DOT_ERR_INVALID_ARG = -1
DOT_ERR_OOM = -2
DOT_ERR_CUDA = -3
DOT_ERR_STEP_LIMIT = -4
DOT_ERR_UNSUPPORTED = -5

DOT_STORAGE_F32, DOT_STORAGE_F16, DOT_STORAGE_BF16 = 0, 1, 2
DOT_ACT_SIGMOID, DOT_ACT_LINEAR = 0, 1
DOT_SIGNAL_NONE, DOT_SIGNAL_SUM_ALPHA, DOT_SIGNAL_MAX_WEIGHT, DOT_SIGNAL_SIGMA = 0, 1, 2, 3
DOT_SELECT_NONE, DOT_SELECT_THRESHOLD, DOT_SELECT_FRACTION, DOT_SELECT_QUANTILE = 0, 1, 2, 3
DOT_MERGE_MEAN, DOT_MERGE_SUM, DOT_MERGE_MAX = 0, 1, 2
DOT_RAYS_BUFFER, DOT_RAYS_CAMERAS = 0, 1
DOT_PRECISION_AUTO, DOT_PRECISION_FAST, DOT_PRECISION_EXACT = 0, 1, 2
DOT_STATUS_STEP_LIMIT = 1
DOT_STATUS_BAD_INPUT = 2

ENTRY_POINTS = ("dot_last_error", "dot_version", "dot_octree_build", "dot_tree_free",
                "dot_tree_get_info", "dot_tree_export", "dot_tree_import", "dot_tree_status",
                "dot_render_forward", "dot_render_backward", "dot_accumulate_signal",
                "dot_select_masks", "dot_refine_plan", "dot_refine_prune", "dot_render_stats",
                "dot_select_masks_noalloc", "dot_render_slots", "dot_mse_grad",
                "dot_rmsprop_step", "dot_compress_sh", "dot_tree_canonicalize",
                "dot_rmsprop_step_sparse", "dot_rmsprop_flush", "dot_render_forward_backward_mse",
                "dot_camera_order", "dot_render_views_host", "dot_render_views_host_workspace",
                "dot_probe_l2_read")

_TORCH_OF_STORAGE = {DOT_STORAGE_F32: torch.float32, DOT_STORAGE_F16: torch.float16,
                     DOT_STORAGE_BF16: torch.bfloat16}
_NP_OF_STORAGE = {DOT_STORAGE_F32: np.float32, DOT_STORAGE_F16: np.float16,
                  DOT_STORAGE_BF16: np.uint16}

P = ctypes.c_void_p


class DotError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdot error {code}: {msg}")
        self.code = code


# ----------------------------------------------------------------------------------------------
# structures
# ----------------------------------------------------------------------------------------------
_ALLOC_FN = ctypes.CFUNCTYPE(P, P, ctypes.c_size_t, P)
_FREE_FN = ctypes.CFUNCTYPE(None, P, P, P)


class dot_allocator(ctypes.Structure):
    _fields_ = [("ctx", P), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


class dot_primitive(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int64), ("p", ctypes.c_int64 * 7)]


class dot_build_desc(ctypes.Structure):
    _fields_ = [("center", ctypes.c_float * 3), ("half_size", ctypes.c_float),
                ("max_depth", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("n_primitives", ctypes.c_int32),
                ("primitives", P), ("density_lo", ctypes.c_float), ("density_hi", ctypes.c_float),
                ("sh_std", ctypes.c_float), ("sh_dc", ctypes.c_float), ("seed", ctypes.c_uint64)]


class dot_tree_info(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("max_level", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("n_coeffs", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("sh_row_stride", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("center", ctypes.c_float * 3), ("half_size", ctypes.c_float),
                ("child", P), ("node_parent", P), ("node_key", P), ("leaf_parent", P),
                ("leaf_key", P), ("sigma", P), ("sh", P), ("palette_bits", ctypes.c_int32),
                ("pad2_", ctypes.c_int32), ("palette", P), ("leaf_record", P), ("rope", P)]


class dot_host_tree(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("sh_degree", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("center", ctypes.c_float * 3), ("half_size", ctypes.c_float),
                ("child", P), ("node_parent", P), ("node_key", P), ("leaf_parent", P),
                ("leaf_key", P), ("sigma", P), ("sh", P)]


class dot_camera(ctypes.Structure):
    _fields_ = [("c2w", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class dot_rays(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_cameras", ctypes.c_int32), ("cameras", P),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("n_rays", ctypes.c_int64),
                ("origins", P), ("dirs", P), ("view_order", P)]


class dot_render_opts(ctypes.Structure):
    _fields_ = [("background", ctypes.c_float * 3), ("eps_T", ctypes.c_float),
                ("color_act", ctypes.c_int32), ("signal_mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("max_steps", ctypes.c_int32)]


class dot_select_opts(ctypes.Structure):
    _fields_ = [("prune_mode", ctypes.c_int32), ("sample_mode", ctypes.c_int32),
                ("prune_value", ctypes.c_double), ("sample_value", ctypes.c_double)]


class dot_refine_counts(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_pruned_groups", ctypes.c_int64), ("n_sampled", ctypes.c_int64),
                ("n_capped", ctypes.c_int64)]


class dot_rmsprop_opts(ctypes.Structure):
    _fields_ = [("lr_sigma", ctypes.c_float), ("lr_sh", ctypes.c_float), ("rho", ctypes.c_float),
                ("eps", ctypes.c_float), ("zero_grad", ctypes.c_int32)]


class dot_leaf_array(ctypes.Structure):
    _fields_ = [("src", P), ("dst", P), ("width", ctypes.c_int32), ("merge", ctypes.c_int32)]


assert ctypes.sizeof(dot_camera) == 72 and ctypes.sizeof(dot_primitive) == 64

# ----------------------------------------------------------------------------------------------
# library loading
# ----------------------------------------------------------------------------------------------
_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libdot (built in-tree first if missing or stale); raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    L = ctypes.CDLL(path)
    L.dot_last_error.restype = ctypes.c_char_p
    L.dot_last_error.argtypes = []
    L.dot_version.restype = ctypes.c_int
    L.dot_version.argtypes = []
    sigs = {
        "dot_octree_build": [ctypes.POINTER(dot_build_desc), ctypes.POINTER(dot_allocator), P, ctypes.POINTER(P)],
        "dot_tree_free": [P],
        "dot_tree_get_info": [P, ctypes.POINTER(dot_tree_info)],
        "dot_tree_export": [P, P, P, P, P, P, P, P, P],
        "dot_tree_import": [ctypes.POINTER(dot_host_tree), ctypes.POINTER(dot_allocator), P, ctypes.POINTER(P)],
        "dot_tree_status": [P, P, ctypes.POINTER(ctypes.c_uint32)],
        "dot_render_forward": [P, ctypes.POINTER(dot_rays), ctypes.POINTER(dot_render_opts), P, P, P, P],
        "dot_render_backward": [P, ctypes.POINTER(dot_rays), ctypes.POINTER(dot_render_opts), P, P, P, P, P, P, P],
        "dot_accumulate_signal": [P, ctypes.POINTER(dot_rays), ctypes.POINTER(dot_render_opts), ctypes.c_int32, P, P],
        "dot_select_masks": [P, P, ctypes.POINTER(dot_select_opts), P, P, P],
        "dot_refine_plan": [P, P, P, ctypes.c_int32, ctypes.POINTER(dot_refine_counts), P],
        "dot_refine_prune": [P, P, P, ctypes.c_int32, P, ctypes.POINTER(dot_leaf_array), ctypes.c_int32, P],
        "dot_render_stats": [P, ctypes.POINTER(dot_rays), ctypes.POINTER(dot_render_opts), ctypes.POINTER(ctypes.c_int64), P],
        "dot_select_masks_noalloc": [P, P, ctypes.POINTER(dot_select_opts), P, P, P],
        "dot_render_slots": [P, ctypes.c_int32, P, ctypes.c_int32, ctypes.POINTER(dot_render_opts), P, P],
        "dot_mse_grad": [P, P, ctypes.c_int64, P, P, P],
        "dot_rmsprop_step": [P, P, P, P, P, ctypes.POINTER(dot_rmsprop_opts), P],
        "dot_compress_sh": [P, ctypes.c_int32, P],
        "dot_tree_canonicalize": [P, P, ctypes.POINTER(dot_leaf_array), ctypes.c_int32, P],
        "dot_rmsprop_step_sparse": [P, P, P, P, P, P, P, ctypes.c_int32, P, ctypes.POINTER(dot_rmsprop_opts), P],
        "dot_rmsprop_flush": [P, P, P, P, ctypes.c_int32, ctypes.POINTER(dot_rmsprop_opts), P],
        "dot_render_forward_backward_mse": [P, ctypes.POINTER(dot_rays), ctypes.POINTER(dot_render_opts),
                                            P, P, P, P, P, P, P, P, P],
        "dot_camera_order": [P, ctypes.c_int32, P],
        "dot_render_views_host": [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P,
                                  ctypes.POINTER(dot_render_opts), P, P, P, ctypes.c_int64, P],
        "dot_probe_l2_read": [P, ctypes.c_int64, ctypes.c_int32, P, P],
    }
    for name, args in sigs.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.dot_render_views_host_workspace.argtypes = [ctypes.c_int32] * 4
    L.dot_render_views_host_workspace.restype = ctypes.c_int64
    _lib = L
    return L


def _check(rc: int):
    if rc != DOT_OK:
        raise DotError(rc, lib().dot_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if isinstance(stream, int) and stream == 0:
        return ctypes.c_void_p(None)            # the legacy default stream
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t: torch.Tensor, dtype, numel=None, name="tensor"):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")


class _CAI:
    """A device buffer exposed through __cuda_array_interface__ (zero-copy torch view)."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "strides": None, "version": 3}
        self._owner = owner


def _view(ptr: int, shape, dtype: torch.dtype, owner) -> torch.Tensor:
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype=dtype, device="cuda")
    ts = {torch.float32: "<f4", torch.float16: "<f2", torch.bfloat16: "<i2", torch.int32: "<i4",
          torch.int64: "<i8", torch.uint8: "|u1"}[dtype]
    t = torch.as_tensor(_CAI(ptr, shape, ts, owner), device="cuda")
    return t.view(torch.bfloat16) if dtype == torch.bfloat16 else t


# ----------------------------------------------------------------------------------------------
# the tree handle
# ----------------------------------------------------------------------------------------------
class TorchAllocator:
    """A dot_allocator whose blocks come from torch's caching allocator: each block is a uint8
    CUDA tensor kept alive until the library frees it (stream-ordered through record_stream).
    ``offset`` shifts every returned pointer by that many bytes inside its tensor (a test hook
    for the library's alignment check).  Keep the object alive while any tree built with it is."""

    def __init__(self, offset: int = 0):
        self.offset = int(offset)
        self.live = {}
        self.n_alloc = self.n_free = 0

        def _alloc(ctx, nbytes, stream):
            try:
                t = torch.empty(int(nbytes) + self.offset, dtype=torch.uint8, device="cuda")
            except RuntimeError:
                return None
            p = t.data_ptr() + self.offset
            self.live[p] = t
            self.n_alloc += 1
            return p

        def _free(ctx, ptr, stream):
            t = self.live.pop(ptr, None)
            if t is not None:
                self.n_free += 1
                if stream:
                    t.record_stream(torch.cuda.ExternalStream(stream))

        self._fns = (_ALLOC_FN(_alloc), _FREE_FN(_free))
        self.struct = dot_allocator(None, self._fns[0], self._fns[1])


class Octree:
    """Owner of a ``dot_tree`` handle.  ``sigma`` / ``sh`` are zero-copy views of the leaf
    parameters (valid until the next refine or free)."""

    def __init__(self, handle: ctypes.c_void_p, allocator: Optional[TorchAllocator] = None):
        self.handle = handle
        self.allocator = allocator        # kept alive for the tree's later allocations and frees

    @property
    def _as_parameter_(self):
        return self.handle

    def info(self) -> dot_tree_info:
        inf = dot_tree_info()
        _check(lib().dot_tree_get_info(self.handle, ctypes.byref(inf)))
        return inf

    @property
    def n_leaves(self) -> int:
        return int(self.info().n_leaves)

    @property
    def n_nodes(self) -> int:
        return int(self.info().n_nodes)

    @property
    def storage(self) -> int:
        return int(self.info().storage)

    @property
    def sh_degree(self) -> int:
        return int(self.info().sh_degree)

    @property
    def sigma(self) -> torch.Tensor:
        inf = self.info()
        return _view(inf.sigma, (inf.n_leaves,), _TORCH_OF_STORAGE[inf.storage], self)

    @property
    def rope(self) -> torch.Tensor:
        """[L, 6] int32 view of the face-neighbour table (read-only; see dot_tree_info)."""
        inf = self.info()
        return _view(inf.rope, (inf.n_leaves, 6), torch.int32, self)

    @property
    def palette_bits(self) -> int:
        return int(self.info().palette_bits)

    @property
    def palette_index(self) -> torch.Tensor:
        """[L] int64 palette row of every leaf of a compressed tree."""
        inf = self.info()
        if not inf.palette_bits:
            raise ValueError("the tree is not compressed")
        rec = _view(inf.leaf_record, (inf.n_leaves,), torch.int32, self)
        return (rec.to(torch.int64) >> 16) & 0xFFFF

    @property
    def palette(self) -> torch.Tensor:
        """[2^bits, 3, K] view of the palette of a compressed tree."""
        inf = self.info()
        if not inf.palette_bits:
            raise ValueError("the tree is not compressed")
        rows = _view(inf.palette, (1 << inf.palette_bits, inf.sh_row_stride),
                     _TORCH_OF_STORAGE[inf.storage], self)
        return rows[:, : 3 * inf.n_coeffs].unflatten(1, (3, inf.n_coeffs))

    @property
    def sh_rows(self) -> torch.Tensor:
        """[L, row_stride] padded rows."""
        inf = self.info()
        if inf.palette_bits:
            raise ValueError("the tree is compressed: see palette and palette_index")
        return _view(inf.sh, (inf.n_leaves, inf.sh_row_stride), _TORCH_OF_STORAGE[inf.storage], self)

    @property
    def sh(self) -> torch.Tensor:
        """[L, 3, K] view of the SH coefficients."""
        inf = self.info()
        K = inf.n_coeffs
        return self.sh_rows[:, : 3 * K].unflatten(1, (3, K))

    def export(self, stream=None) -> dict:
        inf = self.info()
        N, L, K = inf.n_nodes, inf.n_leaves, inf.n_coeffs
        dt = _NP_OF_STORAGE[inf.storage]
        out = {"child": np.empty((N, 8), np.int32), "node_parent": np.empty(N, np.int32),
               "node_key": np.empty(N, np.uint64), "leaf_parent": np.empty(L, np.int32),
               "leaf_key": np.empty(L, np.uint64), "sigma": np.empty(L, dt),
               "sh": np.empty((L, 3, K), dt)}
        _check(lib().dot_tree_export(self.handle, _stream(stream),
                                     *[out[k].ctypes.data_as(P) for k in
                                       ("child", "node_parent", "node_key", "leaf_parent",
                                        "leaf_key", "sigma", "sh")]))
        out.update(center=tuple(inf.center), half_size=float(inf.half_size),
                   sh_degree=int(inf.sh_degree), storage=int(inf.storage),
                   max_level=int(inf.max_level))
        return out

    def status(self, stream=None) -> int:
        s = ctypes.c_uint32(0)
        _check(lib().dot_tree_status(self.handle, _stream(stream), ctypes.byref(s)))
        return int(s.value)

    def free(self):
        if self.handle:
            torch.cuda.synchronize()
            lib().dot_tree_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            if self.handle and _lib is not None:
                _lib.dot_tree_free(self.handle)
                self.handle = None
        except Exception:
            pass


# ----------------------------------------------------------------------------------------------
# descriptors
# ----------------------------------------------------------------------------------------------
def build_desc(center, half_size, max_depth, sh_degree, storage, prims: np.ndarray,
               density=(10.0, 200.0), sh_std=0.5, sh_dc=0.5, seed=0):
    prims = np.ascontiguousarray(prims, dtype=np.int64).reshape(-1, 8)
    d = dot_build_desc()
    d.center = (ctypes.c_float * 3)(*[float(x) for x in center])
    d.half_size = float(half_size)
    d.max_depth = int(max_depth)
    d.sh_degree = int(sh_degree)
    d.storage = int(storage)
    d.n_primitives = prims.shape[0]
    d.primitives = prims.ctypes.data_as(P) if prims.shape[0] else None
    d.density_lo, d.density_hi = float(density[0]), float(density[1])
    d.sh_std, d.sh_dc = float(sh_std), float(sh_dc)
    d.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    d._keep = prims
    return d


def render_opts(background=(1.0, 1.0, 1.0), eps_T=1e-4, color_act=DOT_ACT_SIGMOID,
                signal_mode=DOT_SIGNAL_NONE, precision=DOT_PRECISION_AUTO, max_steps=0):
    o = dot_render_opts()
    o.background = (ctypes.c_float * 3)(*[float(x) for x in background])
    o.eps_T = float(eps_T)
    o.color_act = int(color_act)
    o.signal_mode = int(signal_mode)
    o.precision = int(precision)
    o.max_steps = int(max_steps)
    return o


def rays_buffer(origins: torch.Tensor, dirs: torch.Tensor) -> dot_rays:
    _need(origins, torch.float32, name="origins")
    _need(dirs, torch.float32, origins.numel(), name="dirs")
    r = dot_rays()
    r.kind = DOT_RAYS_BUFFER
    r.n_rays = origins.numel() // 3
    r.origins = _ptr(origins)
    r.dirs = _ptr(dirs)
    r._keep = (origins, dirs)
    return r


def cameras_tensor(cams: Sequence, device="cuda") -> torch.Tensor:
    """float32 [n, 18] device tensor of dot_camera records from seeded_inputs-style cameras."""
    arr = np.stack([c.packed() for c in cams]).astype(np.float32)
    return torch.from_numpy(arr).to(device)


def rays_cameras(cams: torch.Tensor, width: int, height: int,
                 view_order: Optional[torch.Tensor] = None) -> dot_rays:
    """Camera rays of every [n, 18] dot_camera record (device); view_order: optional device
    int32 [n] permutation in which the views are rendered (ray ids unchanged)."""
    _need(cams, torch.float32, name="cameras")
    if cams.dim() != 2 or cams.shape[1] != 18:
        raise ValueError("cameras must be [n, 18] float32 records")
    r = dot_rays()
    r.kind = DOT_RAYS_CAMERAS
    r.n_cameras = cams.shape[0]
    r.cameras = _ptr(cams)
    r.width, r.height = int(width), int(height)
    r.n_rays = 0
    if view_order is not None:
        _need(view_order, torch.int32, cams.shape[0], "view_order")
        r.view_order = _ptr(view_order)
    r._keep = (cams, view_order)
    return r


def dot_camera_order(cams_host: np.ndarray) -> np.ndarray:
    """Nearest-neighbour chain order of the cameras ([n, 18] float32 host records)."""
    c = np.ascontiguousarray(cams_host, dtype=np.float32).reshape(-1, 18)
    order = np.zeros(c.shape[0], np.int32)
    _check(lib().dot_camera_order(c.ctypes.data_as(P), c.shape[0], order.ctypes.data_as(P)))
    return order


def _host(t, dtype, numel=None, name="tensor"):
    """A contiguous CPU tensor of `dtype` (and `numel` elements when given); numpy arrays are
    wrapped without a copy."""
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(t)
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous host {dtype} tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return t


def dot_render_views_host_workspace(n_cameras: int, width: int, height: int,
                                    with_T: bool = False) -> int:
    """Device workspace bytes dot_render_views_host needs (-1 for invalid sizes)."""
    return int(lib().dot_render_views_host_workspace(int(n_cameras), int(width), int(height),
                                                     int(bool(with_T))))


def dot_render_views_host(tree: Octree, cams_host, width: int, height: int,
                          opts: dot_render_opts, rgb_host, T_host=None, view_order=None,
                          workspace: Optional[torch.Tensor] = None, stream=None):
    """Whole views from host cameras ([n, 18] float32 records) to host images (float32
    [n][H][W][3], and [n][H][W] for T_host), chunked with the device-to-host copies overlapping
    the march (see dot.h).  view_order: host int32 [n] permutation or None; workspace: device
    uint8 tensor of at least dot_render_views_host_workspace(...) bytes (allocated when None)."""
    cams = _host(cams_host, torch.float32, name="cameras")
    if cams.dim() != 2 or cams.shape[1] != 18:
        raise ValueError("cameras must be [n, 18] float32 records")
    n = cams.shape[0]
    R = n * int(width) * int(height)
    rgb = _host(rgb_host, torch.float32, 3 * R, "rgb")
    T = _host(T_host, torch.float32, R, "T_final") if T_host is not None else None
    order = None
    if view_order is not None:
        order = _host(view_order, torch.int32, n, "view_order")
    need = dot_render_views_host_workspace(n, width, height, T is not None)
    if need < 0:
        raise ValueError("camera count or resolution out of range")
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device="cuda")
    _need(workspace, torch.uint8, name="workspace")
    _check(lib().dot_render_views_host(tree.handle, _ptr(cams), n, int(width), int(height),
                                       _ptr(order), ctypes.byref(opts), _ptr(rgb), _ptr(T),
                                       _ptr(workspace), workspace.numel(), _stream(stream)))


def n_rays_of(r: dot_rays) -> int:
    if r.kind == DOT_RAYS_BUFFER:
        return int(r.n_rays)
    return int(r.n_cameras) * int(r.width) * int(r.height)


def select_opts(prune_mode=DOT_SELECT_NONE, prune_value=0.0, sample_mode=DOT_SELECT_NONE,
                sample_value=0.0):
    o = dot_select_opts()
    o.prune_mode, o.sample_mode = int(prune_mode), int(sample_mode)
    o.prune_value, o.sample_value = float(prune_value), float(sample_value)
    return o


# ----------------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ----------------------------------------------------------------------------------------------
def dot_version() -> int:
    return int(lib().dot_version())


def dot_last_error() -> str:
    return lib().dot_last_error().decode()


def dot_octree_build(desc: dot_build_desc, stream=None,
                     allocator: Optional[TorchAllocator] = None) -> Octree:
    h = ctypes.c_void_p()
    al = ctypes.byref(allocator.struct) if allocator is not None else None
    _check(lib().dot_octree_build(ctypes.byref(desc), al, _stream(stream), ctypes.byref(h)))
    return Octree(h, allocator)


def dot_tree_import(host: dict, stream=None, allocator: Optional[TorchAllocator] = None) -> Octree:
    """Tree from host arrays (keys child, node_parent, node_key, leaf_parent, leaf_key, sigma,
    sh [L,3,K], center, half_size, sh_degree, storage)."""
    keep = {k: np.ascontiguousarray(host[k]) for k in
            ("child", "node_parent", "node_key", "leaf_parent", "leaf_key", "sigma", "sh")}
    h = dot_host_tree()
    h.n_nodes = keep["node_key"].shape[0]
    h.n_leaves = keep["leaf_key"].shape[0]
    h.sh_degree = int(host["sh_degree"])
    h.storage = int(host["storage"])
    h.center = (ctypes.c_float * 3)(*[float(x) for x in host["center"]])
    h.half_size = float(host["half_size"])
    for k, v in keep.items():
        setattr(h, k, v.ctypes.data_as(P))
    out = ctypes.c_void_p()
    al = ctypes.byref(allocator.struct) if allocator is not None else None
    _check(lib().dot_tree_import(ctypes.byref(h), al, _stream(stream), ctypes.byref(out)))
    return Octree(out, allocator)


def dot_render_forward(tree: Octree, rays: dot_rays, opts: dot_render_opts, rgb: torch.Tensor,
                       T_final: Optional[torch.Tensor] = None,
                       signal: Optional[torch.Tensor] = None, stream=None):
    R = n_rays_of(rays)
    _need(rgb, torch.float32, 3 * R, "rgb")
    if T_final is not None:
        _need(T_final, torch.float32, R, "T_final")
    if signal is not None:
        _need(signal, torch.float32, tree.n_leaves, "signal")
    _check(lib().dot_render_forward(tree.handle, ctypes.byref(rays), ctypes.byref(opts), _ptr(rgb),
                                    _ptr(T_final), _ptr(signal), _stream(stream)))


def dot_render_backward(tree: Octree, rays: dot_rays, opts: dot_render_opts,
                        grad_rgb: torch.Tensor, rgb: torch.Tensor, grad_sigma: torch.Tensor,
                        grad_sh: torch.Tensor, signal: Optional[torch.Tensor] = None,
                        touched: Optional[torch.Tensor] = None, stream=None):
    R = n_rays_of(rays)
    inf = tree.info()
    _need(grad_rgb, torch.float32, 3 * R, "grad_rgb")
    _need(rgb, torch.float32, 3 * R, "rgb")
    _need(grad_sigma, torch.float32, inf.n_leaves, "grad_sigma")
    _need(grad_sh, torch.float32, inf.n_leaves * 3 * inf.n_coeffs, "grad_sh")
    if signal is not None:
        _need(signal, torch.float32, inf.n_leaves, "signal")
    if touched is not None:
        _need(touched, torch.uint8, inf.n_leaves, "touched")
    _check(lib().dot_render_backward(tree.handle, ctypes.byref(rays), ctypes.byref(opts),
                                     _ptr(grad_rgb), _ptr(rgb), _ptr(grad_sigma), _ptr(grad_sh),
                                     _ptr(signal), _ptr(touched), _stream(stream)))


def dot_render_forward_backward_mse(tree: Octree, rays: dot_rays, opts: dot_render_opts,
                                    target: torch.Tensor, rgb: torch.Tensor,
                                    grad_rgb: torch.Tensor, grad_sigma: torch.Tensor,
                                    grad_sh: torch.Tensor, loss_sum: Optional[torch.Tensor] = None,
                                    signal: Optional[torch.Tensor] = None,
                                    touched: Optional[torch.Tensor] = None, stream=None):
    """Forward, MSE gradient and backward of a ray batch in one launch (see dot.h)."""
    R = n_rays_of(rays)
    inf = tree.info()
    for t, n in ((target, "target"), (rgb, "rgb"), (grad_rgb, "grad_rgb")):
        _need(t, torch.float32, 3 * R, n)
    _need(grad_sigma, torch.float32, inf.n_leaves, "grad_sigma")
    _need(grad_sh, torch.float32, inf.n_leaves * 3 * inf.n_coeffs, "grad_sh")
    if loss_sum is not None:
        _need(loss_sum, torch.float64, 1, "loss_sum")
    if signal is not None:
        _need(signal, torch.float32, inf.n_leaves, "signal")
    if touched is not None:
        _need(touched, torch.uint8, inf.n_leaves, "touched")
    _check(lib().dot_render_forward_backward_mse(
        tree.handle, ctypes.byref(rays), ctypes.byref(opts), _ptr(target), _ptr(rgb),
        _ptr(grad_rgb), _ptr(loss_sum), _ptr(grad_sigma), _ptr(grad_sh), _ptr(signal),
        _ptr(touched), _stream(stream)))


def dot_accumulate_signal(tree: Octree, rays: Optional[dot_rays], opts: dot_render_opts,
                          mode: int, signal: torch.Tensor, stream=None):
    _need(signal, torch.float32, tree.n_leaves, "signal")
    rp = ctypes.byref(rays) if rays is not None else None
    _check(lib().dot_accumulate_signal(tree.handle, rp, ctypes.byref(opts), int(mode),
                                       _ptr(signal), _stream(stream)))


def dot_select_masks(tree: Octree, signal: torch.Tensor, opts: dot_select_opts,
                     prune_mark: torch.Tensor, sample_mark: torch.Tensor, stream=None):
    L = tree.n_leaves
    _need(signal, torch.float32, L, "signal")
    _need(prune_mark, torch.uint8, L, "prune_mark")
    _need(sample_mark, torch.uint8, L, "sample_mark")
    _check(lib().dot_select_masks(tree.handle, _ptr(signal), ctypes.byref(opts), _ptr(prune_mark),
                                  _ptr(sample_mark), _stream(stream)))


def dot_select_masks_noalloc(tree: Octree, signal: torch.Tensor, opts: dot_select_opts,
                             prune_mark: torch.Tensor, sample_mark: torch.Tensor, stream=None):
    """dot_select_masks without any device allocation (for callers that must not allocate);
    trees of at most 2^26 leaves, and overlapping calls on one device must be ordered."""
    L = tree.n_leaves
    _need(signal, torch.float32, L, "signal")
    _need(prune_mark, torch.uint8, L, "prune_mark")
    _need(sample_mark, torch.uint8, L, "sample_mark")
    _check(lib().dot_select_masks_noalloc(tree.handle, _ptr(signal), ctypes.byref(opts),
                                          _ptr(prune_mark), _ptr(sample_mark), _stream(stream)))


def dot_refine_plan(tree: Octree, prune_mark: torch.Tensor, sample_mark: torch.Tensor,
                    depth_cap: int, stream=None) -> dict:
    L = tree.n_leaves
    _need(prune_mark, torch.uint8, L, "prune_mark")
    _need(sample_mark, torch.uint8, L, "sample_mark")
    c = dot_refine_counts()
    _check(lib().dot_refine_plan(tree.handle, _ptr(prune_mark), _ptr(sample_mark), int(depth_cap),
                                 ctypes.byref(c), _stream(stream)))
    return {k: int(getattr(c, k)) for k, _ in dot_refine_counts._fields_}


def dot_refine_prune(tree: Octree, prune_mark: torch.Tensor, sample_mark: torch.Tensor,
                     depth_cap: int, leaf_map: torch.Tensor,
                     aux: Sequence = (), stream=None):
    """aux: sequence of (src [L_old, w] f32, dst [L_new, w] f32, merge) tensors / modes."""
    L = tree.n_leaves
    _need(prune_mark, torch.uint8, L, "prune_mark")
    _need(sample_mark, torch.uint8, L, "sample_mark")
    _need(leaf_map, torch.int32, None, "leaf_map")
    arr = (dot_leaf_array * max(1, len(aux)))()
    for i, (src, dst, merge) in enumerate(aux):
        w = src.numel() // L if L else 1
        _need(src, torch.float32, L * w, "aux src")
        _need(dst, torch.float32, None, "aux dst")
        arr[i].src, arr[i].dst, arr[i].width, arr[i].merge = src.data_ptr(), dst.data_ptr(), w, int(merge)
    _check(lib().dot_refine_prune(tree.handle, _ptr(prune_mark), _ptr(sample_mark), int(depth_cap),
                                  _ptr(leaf_map), arr, len(aux), _stream(stream)))


def dot_render_stats(tree: Octree, rays: dot_rays, opts: dot_render_opts, stream=None):
    out = (ctypes.c_int64 * 4)()
    _check(lib().dot_render_stats(tree.handle, ctypes.byref(rays), ctypes.byref(opts), out,
                                  _stream(stream)))
    return {"rays_hit": out[0], "segments": out[1], "occupied": out[2], "child_loads": out[3]}


def dot_render_slots(trees: Sequence[Octree], table: torch.Tensor, max_slots: int,
                     opts: dot_render_opts, work_counter: torch.Tensor, stream=None):
    """One persistent launch over a device slot table (header + max_slots 96-byte slots)."""
    if not (table.is_cuda and table.numel() * table.element_size() >= 16 + 96 * max_slots):
        raise ValueError("table must be a device buffer of 16 + 96 * max_slots bytes")
    if not (work_counter.is_cuda and work_counter.numel() * work_counter.element_size() >= 8):
        raise ValueError("work_counter must be a device buffer of at least 8 bytes")
    handles = (ctypes.c_void_p * len(trees))(*[t.handle.value for t in trees])
    _check(lib().dot_render_slots(handles, len(trees), _ptr(table), int(max_slots),
                                  ctypes.byref(opts), _ptr(work_counter), _stream(stream)))


def rmsprop_opts(lr_sigma=0.1, lr_sh=0.01, rho=0.9, eps=1e-8, zero_grad=True) -> dot_rmsprop_opts:
    """Defaults: the learning rates of Sec. 4.1; rho and eps, which the paper does not give,
    take the usual RMSProp values."""
    o = dot_rmsprop_opts()
    o.lr_sigma, o.lr_sh, o.rho, o.eps = float(lr_sigma), float(lr_sh), float(rho), float(eps)
    o.zero_grad = int(bool(zero_grad))
    return o


def dot_mse_grad(rgb: torch.Tensor, target: torch.Tensor, grad_rgb: torch.Tensor,
                 loss_sum: Optional[torch.Tensor] = None, stream=None):
    """grad_rgb = 2 (rgb - target) / 3R; loss_sum (float64 device scalar) += the MSE."""
    R = rgb.numel() // 3
    _need(rgb, torch.float32, 3 * R, "rgb")
    _need(target, torch.float32, 3 * R, "target")
    _need(grad_rgb, torch.float32, 3 * R, "grad_rgb")
    if loss_sum is not None:
        _need(loss_sum, torch.float64, 1, "loss_sum")
    _check(lib().dot_mse_grad(_ptr(rgb), _ptr(target), R, _ptr(grad_rgb), _ptr(loss_sum),
                              _stream(stream)))


def dot_rmsprop_step(tree: Octree, grad_sigma: torch.Tensor, grad_sh: torch.Tensor,
                     ms_sigma: torch.Tensor, ms_sh: torch.Tensor, opts: dot_rmsprop_opts,
                     stream=None):
    inf = tree.info()
    L, K = inf.n_leaves, inf.n_coeffs
    _need(grad_sigma, torch.float32, L, "grad_sigma")
    _need(ms_sigma, torch.float32, L, "ms_sigma")
    _need(grad_sh, torch.float32, L * 3 * K, "grad_sh")
    _need(ms_sh, torch.float32, L * 3 * K, "ms_sh")
    _check(lib().dot_rmsprop_step(tree.handle, _ptr(grad_sigma), _ptr(grad_sh), _ptr(ms_sigma),
                                  _ptr(ms_sh), ctypes.byref(opts), _stream(stream)))


def dot_rmsprop_step_sparse(tree: Octree, grad_sigma, grad_sh, ms_sigma, ms_sh,
                            touched: torch.Tensor, last_step: torch.Tensor, step: int,
                            work: torch.Tensor, opts: dot_rmsprop_opts, stream=None):
    """RMSProp of the touched leaves only, the decay of the others deferred (see dot.h)."""
    inf = tree.info()
    L, K = inf.n_leaves, inf.n_coeffs
    _need(grad_sigma, torch.float32, L, "grad_sigma")
    _need(ms_sigma, torch.float32, L, "ms_sigma")
    _need(grad_sh, torch.float32, L * 3 * K, "grad_sh")
    _need(ms_sh, torch.float32, L * 3 * K, "ms_sh")
    _need(touched, torch.uint8, L, "touched")
    _need(last_step, torch.int32, L, "last_step")
    _need(work, torch.int32, L + 1, "work")
    _check(lib().dot_rmsprop_step_sparse(tree.handle, _ptr(grad_sigma), _ptr(grad_sh),
                                         _ptr(ms_sigma), _ptr(ms_sh), _ptr(touched),
                                         _ptr(last_step), int(step), _ptr(work),
                                         ctypes.byref(opts), _stream(stream)))


def dot_rmsprop_flush(tree: Octree, ms_sigma, ms_sh, last_step: torch.Tensor, step: int,
                      opts: dot_rmsprop_opts, stream=None):
    inf = tree.info()
    L, K = inf.n_leaves, inf.n_coeffs
    _need(ms_sigma, torch.float32, L, "ms_sigma")
    _need(ms_sh, torch.float32, L * 3 * K, "ms_sh")
    _need(last_step, torch.int32, L, "last_step")
    _check(lib().dot_rmsprop_flush(tree.handle, _ptr(ms_sigma), _ptr(ms_sh), _ptr(last_step),
                                   int(step), ctypes.byref(opts), _stream(stream)))


def dot_compress_sh(tree: Octree, bits: int, stream=None):
    """Median-cut palette of 2^bits SH rows (the compressed model of Sec. 4.1); synchronises."""
    _check(lib().dot_compress_sh(tree.handle, int(bits), _stream(stream)))


def dot_tree_canonicalize(tree: Octree, leaf_perm: torch.Tensor, aux: Sequence = (),
                          stream=None):
    """Renumbers the tree in canonical (breadth-first Morton) order; leaf_perm [L] int32 receives
    the old id of every new leaf; aux: (src [L, w] f32, dst [L, w] f32) pairs permuted alike."""
    L = tree.n_leaves
    _need(leaf_perm, torch.int32, L, "leaf_perm")
    arr = (dot_leaf_array * max(1, len(aux)))()
    for i, (src, dst) in enumerate(aux):
        w = src.numel() // L if L else 1
        _need(src, torch.float32, L * w, "aux src")
        _need(dst, torch.float32, L * w, "aux dst")
        arr[i].src, arr[i].dst, arr[i].width, arr[i].merge = src.data_ptr(), dst.data_ptr(), w, 0
    _check(lib().dot_tree_canonicalize(tree.handle, _ptr(leaf_perm), arr, len(aux), _stream(stream)))


def dot_tree_status(tree: Octree, stream=None) -> int:
    return tree.status(stream)


def dot_probe_l2_read(buf: torch.Tensor, passes: int, sink: Optional[torch.Tensor] = None,
                      stream=None):
    """Streams the device buffer `passes` times with L2-only loads (a bandwidth measurement)."""
    if not buf.is_cuda:
        raise ValueError("buf must be a device tensor")
    nbytes = buf.numel() * buf.element_size()
    _check(lib().dot_probe_l2_read(_ptr(buf), nbytes, int(passes), _ptr(sink), _stream(stream)))
