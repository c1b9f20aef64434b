"""FP64 CPU oracle of the Dynamic PlenOctree (DOT) hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
package.  The product path (``paper_2307_15333_gb300``) never imports, links or executes it, and
the two share no code; the only common module is ``seeded_inputs`` (input generation only).

The C source (``oracle.c``) is plain FP64 code following the paper's definitions: the octree of
Sec. 3 (Preliminaries), the volume rendering of Eq. 1-2, the training signal of Sec. 3.1, the
thresholds / top-k of Sec. 3.2 and Algorithm 1, and the prune (Eq. 3) and sample (Eq. 4)
operations.  This module compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ACT_SIGMOID = 0
ACT_LINEAR = 1
SIGNAL_NONE = 0
SIGNAL_SUM_ALPHA = 1
SIGNAL_MAX_WEIGHT = 2
SELECT_NONE = 0
SELECT_THRESHOLD = 1
SELECT_FRACTION = 2
SELECT_QUANTILE = 3


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, FP64, no FP contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                               "-fopenmp", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _OTree(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("child", ctypes.c_void_p), ("node_parent", ctypes.c_void_p),
                ("node_key", ctypes.c_void_p), ("leaf_parent", ctypes.c_void_p),
                ("leaf_key", ctypes.c_void_p), ("leaf_inside", ctypes.c_void_p)]


class _OOpts(ctypes.Structure):
    _fields_ = [("root_lo", ctypes.c_double * 3), ("root_size", ctypes.c_double),
                ("sh_degree", ctypes.c_int32), ("color_act", ctypes.c_int32),
                ("bg", ctypes.c_double * 3), ("eps_T", ctypes.c_double)]


class _Counts(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_leaves", ctypes.c_int64),
                ("n_pruned_groups", ctypes.c_int64), ("n_sampled", ctypes.c_int64),
                ("n_capped", ctypes.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            L.oracle_build.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_OTree)]
            L.oracle_tree_free.argtypes = [ctypes.POINTER(_OTree)]
            L.oracle_segments.argtypes = [ctypes.POINTER(_OTree), ctypes.POINTER(_OOpts), P, P,
                                          ctypes.c_int64, P, P, P]
            L.oracle_segments.restype = ctypes.c_int64
            L.oracle_sh_basis.argtypes = [ctypes.c_int32, P, P]
            L.oracle_render.argtypes = [ctypes.POINTER(_OTree), ctypes.POINTER(_OOpts), P, P,
                                        ctypes.c_int64, P, P, P, P, P, ctypes.c_int32, P, P,
                                        ctypes.c_int32]
            L.oracle_backward.argtypes = [ctypes.POINTER(_OTree), ctypes.POINTER(_OOpts), P, P,
                                          ctypes.c_int64, P, P, P, P, P, P, P]
            L.oracle_select.argtypes = [P, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                        ctypes.c_int32, ctypes.c_double, P, P]
            L.oracle_refine.argtypes = [ctypes.POINTER(_OTree), P, P, ctypes.c_int32, P, P,
                                        ctypes.c_int32, ctypes.POINTER(_OTree),
                                        ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(_Counts)]
            L.oracle_mse.argtypes = [ctypes.c_int64, P, P, P]
            L.oracle_mse.restype = ctypes.c_double
            L.oracle_rmsprop.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double]
            L.oracle_median_cut.argtypes = [ctypes.c_int64, ctypes.c_int32, P, ctypes.c_int32,
                                            P, P]
            L.oracle_free.argtypes = [P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _copy_out(t: _OTree) -> dict:
    N, L = t.n_nodes, t.n_leaves

    def arr(p, n, dt):
        if n == 0:
            return np.zeros(0, dtype=dt)
        buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(p)
        return np.frombuffer(buf, dtype=dt).copy()

    return {
        "child": arr(t.child, N * 8, np.int32).reshape(N, 8),
        "node_parent": arr(t.node_parent, N, np.int32),
        "node_key": arr(t.node_key, N, np.uint64),
        "leaf_parent": arr(t.leaf_parent, L, np.int32),
        "leaf_key": arr(t.leaf_key, L, np.uint64),
        "leaf_inside": arr(t.leaf_inside, L, np.uint8),
    }


def _as_otree(tree: dict):
    keep = {k: np.ascontiguousarray(v) for k, v in tree.items()}
    ot = _OTree(keep["node_key"].shape[0], keep["leaf_key"].shape[0],
                _ptr(keep["child"]), _ptr(keep["node_parent"]), _ptr(keep["node_key"]),
                _ptr(keep["leaf_parent"]), _ptr(keep["leaf_key"]),
                _ptr(keep.get("leaf_inside", np.zeros(keep["leaf_key"].shape[0], np.uint8))))
    return ot, keep


def _opts(root_lo, root_size, sh_degree=0, color_act=ACT_SIGMOID, bg=(1.0, 1.0, 1.0),
          eps_T=1e-4):
    return _OOpts((ctypes.c_double * 3)(*[float(x) for x in root_lo]), float(root_size),
                  int(sh_degree), int(color_act), (ctypes.c_double * 3)(*[float(x) for x in bg]),
                  float(eps_T))


def build_tree(prims: np.ndarray, max_depth: int) -> dict:
    """Octree of the primitive union (the root is always subdivided; a cell is subdivided while it
    meets a primitive and its level is below max_depth), canonical BFS / Morton numbering."""
    L = lib()
    prims = np.ascontiguousarray(prims, dtype=np.int64)
    t = _OTree()
    rc = L.oracle_build(_ptr(prims), prims.shape[0], int(max_depth), ctypes.byref(t))
    if rc != 0:
        raise ValueError("oracle_build failed")
    out = _copy_out(t)
    L.oracle_tree_free(ctypes.byref(t))
    return out


def scene_tree(scene) -> dict:
    return build_tree(scene.prims, scene.max_depth)


def root_of(scene):
    return scene.root_lo, 2.0 * scene.half_size


def segments(tree: dict, root_lo, root_size, o, d):
    L = lib()
    ot, keep = _as_otree(tree)
    op = _opts(root_lo, root_size)
    o = np.ascontiguousarray(o, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    cap = 64
    while True:
        leaf = np.zeros(cap, np.int32)
        ti = np.zeros(cap, np.float64)
        to = np.zeros(cap, np.float64)
        n = L.oracle_segments(ctypes.byref(ot), ctypes.byref(op), _ptr(o), _ptr(d), cap,
                              _ptr(leaf), _ptr(ti), _ptr(to))
        if n >= 0:
            return leaf[:n], ti[:n], to[:n]
        cap = -n


def sh_basis(deg: int, d) -> np.ndarray:
    Y = np.zeros(16, np.float64)
    dd = np.ascontiguousarray(d, dtype=np.float64)
    lib().oracle_sh_basis(int(deg), _ptr(dd), _ptr(Y))
    return Y[: (deg + 1) ** 2]


def render(tree, root_lo, root_size, sigma, sh, sh_degree, o, d, *, bg=(1.0, 1.0, 1.0),
           eps_T=1e-4, color_act=ACT_SIGMOID, signal=None, signal_mode=SIGNAL_NONE,
           threads=1, margin=False):
    """Eq. 1-2 per ray.  sigma [L] and sh [L,3,K] are float64 copies of the stored values.
    Returns rgb [n,3], T_final [n], segments used per ray [n] (and, with margin=True, each ray's
    closest relative approach of T to eps_T); `signal` is accumulated in place."""
    L = lib()
    ot, keep = _as_otree(tree)
    op = _opts(root_lo, root_size, sh_degree, color_act, bg, eps_T)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    sh = np.ascontiguousarray(sh, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
    n = o.shape[0]
    rgb = np.zeros((n, 3), np.float64)
    Tf = np.zeros(n, np.float64)
    nseg = np.zeros(n, np.int32)
    mg = np.zeros(n, np.float64)
    if signal is not None:
        assert signal.dtype == np.float64 and signal.flags.c_contiguous
    L.oracle_render(ctypes.byref(ot), ctypes.byref(op), _ptr(sigma), _ptr(sh), n, _ptr(o),
                    _ptr(d), _ptr(rgb), _ptr(Tf), _ptr(signal) if signal is not None else None,
                    int(signal_mode), _ptr(nseg), _ptr(mg), int(threads))
    if margin:
        return rgb, Tf, nseg, mg
    return rgb, Tf, nseg


def backward(tree, root_lo, root_size, sigma, sh, sh_degree, o, d, grad_rgb, *,
             bg=(1.0, 1.0, 1.0), eps_T=1e-4, color_act=ACT_SIGMOID):
    """Gradient of sum(grad_rgb * rgb) w.r.t. sigma [L] and sh [L,3,K], plus the per-entry sums
    of the magnitudes of the accumulated terms (the conditioning of each sum)."""
    L = lib()
    ot, keep = _as_otree(tree)
    op = _opts(root_lo, root_size, sh_degree, color_act, bg, eps_T)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    sh = np.ascontiguousarray(sh, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float32).reshape(-1, 3)
    g = np.ascontiguousarray(grad_rgb, dtype=np.float64).reshape(-1, 3)
    gs = np.zeros_like(sigma)
    gsh = np.zeros_like(sh)
    asg = np.zeros_like(sigma)
    ash = np.zeros_like(sh)
    L.oracle_backward(ctypes.byref(ot), ctypes.byref(op), _ptr(sigma), _ptr(sh), o.shape[0],
                      _ptr(o), _ptr(d), _ptr(g), _ptr(gs), _ptr(gsh), _ptr(asg), _ptr(ash))
    return gs, gsh, asg, ash


def select(signal, prune_mode=SELECT_NONE, prune_value=0.0, sample_mode=SELECT_NONE,
           sample_value=0.0):
    s = np.ascontiguousarray(signal, dtype=np.float32)
    n = s.shape[0]
    pm = np.zeros(n, np.uint8)
    sm = np.zeros(n, np.uint8)
    lib().oracle_select(_ptr(s), n, int(prune_mode), float(prune_value), int(sample_mode),
                        float(sample_value), _ptr(pm), _ptr(sm))
    return pm, sm


def refine(tree, sigma, sh, prune_mark, sample_mark, d_cap):
    """Prune (Eq. 3) and sample (Eq. 4).  sigma [L] and sh [L,...] float64.  Returns
    (new_tree, leaf_map, sigma_new, sh_new, counts) with FP64 merged means."""
    L = lib()
    ot, keep = _as_otree(tree)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    sh = np.ascontiguousarray(sh, dtype=np.float64)
    nl = sigma.shape[0]
    n_sh = int(np.prod(sh.shape[1:])) if sh.ndim > 1 else 1
    pm = np.ascontiguousarray(prune_mark, dtype=np.uint8)
    sm = np.ascontiguousarray(sample_mark, dtype=np.uint8)
    out = _OTree()
    lm_p, so_p, sho_p = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    cnt = _Counts()
    L.oracle_refine(ctypes.byref(ot), _ptr(sigma), _ptr(sh), n_sh, _ptr(pm), _ptr(sm),
                    int(d_cap), ctypes.byref(out), ctypes.byref(lm_p), ctypes.byref(so_p),
                    ctypes.byref(sho_p), ctypes.byref(cnt))
    new = _copy_out(out)
    new.pop("leaf_inside")
    n_new = out.n_leaves

    def take(p, n, dt):
        if n == 0:
            return np.zeros(0, dt)
        buf = (ctypes.c_char * (n * np.dtype(dt).itemsize)).from_address(p.value)
        return np.frombuffer(buf, dtype=dt).copy()

    lm = take(lm_p, n_new, np.int32)
    so = take(so_p, n_new, np.float64)
    sho = take(sho_p, n_new * n_sh, np.float64).reshape((n_new,) + tuple(sh.shape[1:]))
    L.oracle_tree_free(ctypes.byref(out))
    for p in (lm_p, so_p, sho_p):
        L.oracle_free(p)
    counts = {k: getattr(cnt, k) for k, _ in _Counts._fields_}
    return new, lm, so, sho, counts


def mse(rgb, target):
    """Loss and gradient of the MSE of Algorithm 1 (optimization) over rays x 3 channels."""
    rgb = np.ascontiguousarray(rgb, dtype=np.float64).reshape(-1, 3)
    target = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 3)
    grad = np.zeros_like(rgb)
    loss = lib().oracle_mse(rgb.shape[0], _ptr(rgb), _ptr(target), _ptr(grad))
    return loss, grad


def rmsprop(param, ms, grad, lr, rho, eps):
    """One RMSProp step (Sec. 3.3) on copies: returns (param_new, ms_new), float64."""
    p = np.array(param, dtype=np.float64, copy=True, order="C")
    m = np.array(ms, dtype=np.float64, copy=True, order="C")
    g = np.ascontiguousarray(grad, dtype=np.float64)
    assert p.size == m.size == g.size
    lib().oracle_rmsprop(p.size, _ptr(p), _ptr(m), _ptr(g), float(lr), float(rho), float(eps))
    return p, m


def remap_leaf_values(old_tree, leaf_map, values, merge="mean"):
    """Per-leaf values carried through a refine: a surviving or copied leaf takes its source
    leaf's value; a merged parent (leaf_map = -1 - p) the mean, sum or max of its 8 children's
    (Eq. 3 for the mean).  values [L_old, ...] float64 -> [L_new, ...]."""
    v = np.asarray(values, dtype=np.float64)
    out = np.empty((len(leaf_map),) + v.shape[1:], np.float64)
    child = old_tree["child"]
    for u, m in enumerate(leaf_map):
        if m >= 0:
            out[u] = v[m]
            continue
        kids = v[[-1 - c for c in child[-1 - m]]]
        if merge == "max":
            out[u] = kids.max(axis=0)
        elif merge == "sum":
            out[u] = kids.sum(axis=0)
        else:
            out[u] = kids.mean(axis=0)
    return out


def prune_recursive(tree, sigma, sh, signal, tau, d_cap, recursive=True, merge="sum", aux=()):
    """Algorithm 1's pruning: merge every group whose 8 leaves all have signal <= tau (Sec. 3.2
    threshold), and, when recursive, repeat on the merged tree -- a merged parent's signal being
    the sum (or max) of its children's -- until no group qualifies.  aux: per-leaf arrays carried
    along as means.  Returns (tree, sigma, sh, signal, aux, passes)."""
    aux = [np.asarray(a, np.float64) for a in aux]
    passes = []
    while True:
        pm, _ = select(signal, SELECT_THRESHOLD, tau)
        sm = np.zeros_like(pm)
        new, lm, so, sho, cnt = refine(tree, sigma, sh, pm, sm, d_cap)
        if cnt["n_pruned_groups"] == 0:
            break
        signal = remap_leaf_values(tree, lm, signal, merge)
        aux = [remap_leaf_values(tree, lm, a, "mean") for a in aux]
        tree, sigma, sh = new, so, sho
        passes.append(cnt)
        if not recursive:
            break
    return tree, sigma, sh, signal, aux, passes


def median_cut(x, bits):
    """Median-cut quantisation (Sec. 4.1, compressed models) of the rows of x [n, dim] into
    2^bits boxes: returns (index [n] int32, palette [2^bits, dim] float64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, dim = x.shape
    index = np.zeros(n, np.int32)
    pal = np.zeros((1 << bits, dim), np.float64)
    rc = lib().oracle_median_cut(n, dim, _ptr(x), int(bits), _ptr(index), _ptr(pal))
    assert rc == 0
    return index, pal


def canonicalize(tree, leaf_values=()):
    """The canonical numbering of a tree's cells (the build's order: breadth first, Morton order
    within a level), which is ascending key order since a key is 1 << 3l | morton code.  Nodes and
    leaves are sorted by key (a library sort); child pointers and parents follow.  Returns
    (new_tree, perm) with perm[new leaf] = old leaf, and the leaf_values arrays permuted."""
    nk = np.asarray(tree["node_key"], np.uint64)
    lk = np.asarray(tree["leaf_key"], np.uint64)
    nperm = np.argsort(nk, kind="stable")
    lperm = np.argsort(lk, kind="stable")
    n_new = np.empty(nk.size, np.int64)
    n_new[nperm] = np.arange(nk.size)
    l_new = np.empty(lk.size, np.int64)
    l_new[lperm] = np.arange(lk.size)
    old_child = np.asarray(tree["child"], np.int64)[nperm]
    child = np.where(old_child >= 0, n_new[np.maximum(old_child, 0)],
                     -1 - l_new[np.maximum(-1 - old_child, 0)]).astype(np.int32)
    npar = np.asarray(tree["node_parent"], np.int64)[nperm]
    node_parent = np.where(npar >= 0, n_new[np.maximum(npar, 0)], -1).astype(np.int32)
    leaf_parent = n_new[np.asarray(tree["leaf_parent"], np.int64)[lperm]].astype(np.int32)
    new = {"n_nodes": nk.size, "n_leaves": lk.size, "child": child, "node_parent": node_parent,
           "node_key": nk[nperm], "leaf_parent": leaf_parent, "leaf_key": lk[lperm]}
    vals = [np.asarray(v)[lperm] for v in leaf_values]
    return new, lperm.astype(np.int32), vals


def key_level(keys) -> np.ndarray:
    """Level of each Morton key with a leading 1 bit (reads the key format, no method logic)."""
    k = np.asarray(keys, dtype=np.uint64)
    bl = np.zeros(k.shape, np.int64)
    x = k.copy()
    while np.any(x):
        nz = x != 0
        bl[nz] += 1
        x = x >> np.uint64(1)
    return (bl - 1) // 3
