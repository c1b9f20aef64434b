"""Seeded synthetic inputs shared by the FP64 oracle, the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the rendering method.  It produces:

* scenes: primitive lists (spheres, axis-aligned boxes, vertical cylinders, ground slabs) quantised
  to integer multiples of 2^-24 of the root-cube edge, plus the leaf-parameter distribution;
* pinhole cameras and their float32 rays, built by a fixed sequence of IEEE round-to-nearest-even
  float32 operations so that any implementation that performs the same operations obtains the same
  bits;
* leaf parameters drawn by a counter-based generator (SplitMix64, Steele, Lea and Flood, OOPSLA
  2014) keyed by the leaf's Morton key, so that the draw does not depend on the leaf numbering;
* random ray batches, gradients, signals and masks for the parity tests.

The workloads stand in for the NeRF-synthetic and Tanks & Temples scenes of the paper (Sec. 4.1),
which are not available: sizes, resolutions, view counts, SH degrees and depths follow the paper's
setup (512^3 grid, 16 / 4 SH components, 800x800 and 1920x1080 views).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

Q_BITS = 24
Q = 1 << Q_BITS                      # quantisation grid of primitive parameters per root edge

PRIM_SPHERE = 0                      # p = (cx, cy, cz, r)
PRIM_BOX = 1                         # p = (lox, loy, loz, hix, hiy, hiz)
PRIM_CYLINDER = 2                    # p = (cx, cz, r, y0, y1), axis along +y (up)

STORAGE_F32 = 0
STORAGE_F16 = 1
STORAGE_BF16 = 2
STORAGE_NAMES = {STORAGE_F32: "f32", STORAGE_F16: "f16", STORAGE_BF16: "bf16"}


@dataclasses.dataclass
class Scene:
    """A synthetic scene: root cube, depth, primitives and the leaf-parameter distribution."""
    name: str
    center: Tuple[float, float, float]
    half_size: float
    max_depth: int
    sh_degree: int
    storage: int
    prims: np.ndarray                  # int64 [n, 8]: type, p0..p6 in units of 2^-24 root edge
    density_lo: float
    density_hi: float
    sh_std: float
    sh_dc: float
    seed: int

    @property
    def n_coeffs(self) -> int:
        return (self.sh_degree + 1) ** 2

    @property
    def root_lo(self) -> np.ndarray:
        return np.array(self.center, dtype=np.float64) - self.half_size


# ----------------------------------------------------------------------------------------------
# primitive quantisation
# ----------------------------------------------------------------------------------------------

def _q(v: float) -> int:
    return int(round(v * Q))


def _to_unit(x, center, half):
    return (np.asarray(x, dtype=np.float64) - (np.asarray(center, dtype=np.float64) - half)) / (2.0 * half)


def sphere(c_world, r_world, center, half) -> List[int]:
    u = _to_unit(c_world, center, half)
    return [PRIM_SPHERE, _q(u[0]), _q(u[1]), _q(u[2]), _q(r_world / (2 * half)), 0, 0, 0]


def box(lo_world, hi_world, center, half) -> List[int]:
    a = _to_unit(lo_world, center, half)
    b = _to_unit(hi_world, center, half)
    return [PRIM_BOX, _q(a[0]), _q(a[1]), _q(a[2]), _q(b[0]), _q(b[1]), _q(b[2]), 0]


def cylinder(cx_world, cz_world, r_world, y0_world, y1_world, center, half) -> List[int]:
    c = _to_unit([cx_world, y0_world, cz_world], center, half)
    y1 = _to_unit([0.0, y1_world, 0.0], center, half)[1]
    return [PRIM_CYLINDER, _q(c[0]), _q(c[2]), _q(r_world / (2 * half)), _q(c[1]), _q(y1), 0, 0]


def _prims(rows) -> np.ndarray:
    return np.ascontiguousarray(np.array(rows, dtype=np.int64).reshape(-1, 8))


# ----------------------------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------------------------

def tiny_sphere_scene(seed: int = 0, max_depth: int = 4, sh_degree: int = 1,
                      storage: int = STORAGE_F32) -> Scene:
    """Tiny plain-render scene: root [-1,1]^3, one sphere of radius 0.4, centre ~ U[-0.3,0.3]^3.

    sigma ~ U(5, 50) in the finest cells meeting the sphere; SH ~ N(0, 0.3) with no DC offset.
    """
    rng = np.random.default_rng(seed)
    c = rng.uniform(-0.3, 0.3, size=3)
    center, half = (0.0, 0.0, 0.0), 1.0
    prims = _prims([sphere(c, 0.4, center, half)])
    return Scene("tiny_sphere", center, half, max_depth, sh_degree, storage, prims,
                 5.0, 50.0, 0.3, 0.0, seed)


def nerf_synthetic_scene(seed: int = 1000, max_depth: int = 9, sh_degree: int = 3,
                         storage: int = STORAGE_F16) -> Scene:
    """NeRF-synthetic-shaped scene: seeded union of 8 spheres/boxes in [-1.5,1.5]^3.

    Sphere radii ~ U(0.15, 0.40), box half-extents ~ U(0.10, 0.33) per axis, centres ~
    U[-0.9,0.9]^3.  The ranges were chosen once so that the depth-9 (512^3) octree has 2-4 M leaves.
    sigma ~ U(10, 200) inside, SH ~ N(0, 0.5) with DC offset 0.5, FP16 storage.
    """
    rng = np.random.default_rng(seed)
    center, half = (0.0, 0.0, 0.0), 1.5
    rows = []
    for _ in range(8):
        kind = rng.integers(0, 2)
        c = rng.uniform(-0.9, 0.9, size=3)
        if kind == 0:
            rows.append(sphere(c, rng.uniform(0.15, 0.40), center, half))
        else:
            he = rng.uniform(0.10, 0.33, size=3)
            rows.append(box(c - he, c + he, center, half))
    return Scene("nerf_synthetic", center, half, max_depth, sh_degree, storage, _prims(rows),
                 10.0, 200.0, 0.5, 0.5, seed)


def tanks_temples_scene(seed: int = 3000, max_depth: int = 10, sh_degree: int = 3,
                        storage: int = STORAGE_BF16) -> Scene:
    """Tanks&Temples-shaped large scene: 64 primitives in [-3,3]^3 (boxes, vertical cylinders,
    one ground slab), depth 10 (1024^3), BF16 leaves; ranges chosen once for 8-12 M leaves.
    Box half-extents ~ U(0.05, 0.2), cylinder radii ~ U(0.04, 0.12), heights ~ U(0.2, 1.2)."""
    rng = np.random.default_rng(seed)
    center, half = (0.0, 0.0, 0.0), 3.0
    rows = [box((-2.6, -1.025, -2.6), (2.6, -1.0, 2.6), center, half)]    # ground slab
    for _ in range(63):
        kind = rng.integers(0, 2)
        x, z = rng.uniform(-2.2, 2.2, size=2)
        if kind == 0:
            he = rng.uniform(0.05, 0.2, size=3)
            y = -1.0 + he[1] + rng.uniform(0.0, 0.6)
            c = np.array([x, y, z])
            rows.append(box(c - he, c + he, center, half))
        else:
            r = rng.uniform(0.04, 0.12)
            hgt = rng.uniform(0.2, 1.2)
            rows.append(cylinder(x, z, r, -1.0, -1.0 + hgt, center, half))
    return Scene("tanks_temples", center, half, max_depth, sh_degree, storage, _prims(rows),
                 10.0, 200.0, 0.5, 0.5, seed)


def box_scene(lo, hi, *, center=(0.0, 0.0, 0.0), half=1.0, max_depth=3, sh_degree=0,
              storage=STORAGE_F32, density=(5.0, 50.0), sh_std=0.3, sh_dc=0.0, seed=7) -> Scene:
    """One axis-aligned box; used for closed-form and hand-checked cases."""
    return Scene("box", center, half, max_depth, sh_degree, storage,
                 _prims([box(lo, hi, center, half)]), density[0], density[1], sh_std, sh_dc, seed)


def random_scene(seed: int, *, max_depth=4, sh_degree=2, storage=STORAGE_F32, n_prims=3,
                 half=1.0) -> Scene:
    """A few random primitives of every type; used for small parity and edge cases."""
    rng = np.random.default_rng(seed)
    center = (0.0, 0.0, 0.0)
    rows = []
    for _ in range(n_prims):
        kind = int(rng.integers(0, 3))
        c = rng.uniform(-0.7 * half, 0.7 * half, size=3)
        if kind == 0:
            rows.append(sphere(c, rng.uniform(0.1, 0.35) * half, center, half))
        elif kind == 1:
            he = rng.uniform(0.05, 0.3, size=3) * half
            rows.append(box(c - he, c + he, center, half))
        else:
            rows.append(cylinder(c[0], c[2], rng.uniform(0.05, 0.25) * half, c[1] - 0.3 * half,
                                 c[1] + 0.3 * half, center, half))
    return Scene(f"random{seed}", center, half, max_depth, sh_degree, storage, _prims(rows),
                 5.0, 60.0, 0.4, 0.2, seed)


# ----------------------------------------------------------------------------------------------
# counter-based generator and leaf parameters
# ----------------------------------------------------------------------------------------------

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """Output number `counter` (0-based) of SplitMix64 seeded with `seed`.

    SplitMix64 advances its state by the golden gamma 0x9E3779B97F4A7C15 and returns the
    finaliser mix(state) (variant 13 of Stafford's mixer); output n is therefore
    mix(seed + (n + 1) * gamma) modulo 2^64.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def irwin_hall_scale(sh_std: float) -> np.float32:
    """float32 factor turning the centred Irwin-Hall integer (see leaf_params) into N(0, sh_std)."""
    s_ih = 2.0 * math.sqrt(4.0 * (65536.0 * 65536.0 - 1.0) / 12.0)
    return np.float32(float(np.float32(sh_std)) / s_ih)     # the std as a float32 parameter


def f32_to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest, ties to even); returns uint16 bits."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return b.astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, dtype=np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def round_to_storage(x32: np.ndarray, storage: int) -> np.ndarray:
    """float32 -> stored representation (float32, float16, or uint16 bfloat16 bits)."""
    if storage == STORAGE_F32:
        return np.ascontiguousarray(x32, dtype=np.float32)
    if storage == STORAGE_F16:
        return np.ascontiguousarray(x32, dtype=np.float32).astype(np.float16)
    return f32_to_bf16_bits(x32)


def storage_to_f64(v: np.ndarray, storage: int) -> np.ndarray:
    if storage == STORAGE_BF16:
        return bf16_bits_to_f64(v)
    return np.asarray(v).astype(np.float64)


def leaf_params(leaf_key: np.ndarray, inside: np.ndarray, scene: Scene):
    """Seeded leaf parameters keyed by the leaf's Morton key.

    Component c of a leaf with key k uses the 64-bit draw h = splitmix64(seed, 64*k + c):
      c = 0 (density): inside leaves get sigma = lo + (hi - lo) * u with u = (h >> 40) * 2^-24,
        evaluated as float32 products and sums (round to nearest even); other leaves get 0.
      c = 1 + ch*K + j (SH coefficient j of channel ch): four 16-bit fields of h are summed
        (Irwin-Hall, n = 4), centred as z = 2*sum - 4*65535 (exact in float32), scaled by
        float32(std / std_IH) in float32, and the DC term (j = 0) gets + dc in float32.
    Values are then rounded to the storage type (RNE).  Returns (sigma[L], sh[L, 3, K]) in the
    storage representation (bfloat16 as uint16 bits).
    """
    K = scene.n_coeffs
    keys = np.asarray(leaf_key, dtype=np.uint64)
    L = keys.shape[0]
    base = keys * np.uint64(64)
    f32 = np.float32
    # density
    h0 = splitmix64(scene.seed, base)
    u = (h0 >> np.uint64(40)).astype(np.float32) * f32(2.0 ** -24)
    lo, hi = f32(scene.density_lo), f32(scene.density_hi)
    sig = lo + (hi - lo) * u
    sig = np.where(np.asarray(inside, dtype=bool), sig, f32(0.0)).astype(np.float32)
    # SH
    comp = np.arange(1, 1 + 3 * K, dtype=np.uint64)
    h = splitmix64(scene.seed, base[:, None] + comp[None, :])
    m = np.uint64(0xFFFF)
    s = ((h & m) + ((h >> np.uint64(16)) & m) + ((h >> np.uint64(32)) & m)
         + ((h >> np.uint64(48)) & m)).astype(np.int64)
    z = (2 * s - 4 * 65535).astype(np.float32)
    v = z * irwin_hall_scale(scene.sh_std)
    v = v.reshape(L, 3, K)
    v[:, :, 0] = v[:, :, 0] + f32(scene.sh_dc)
    return round_to_storage(sig, scene.storage), round_to_storage(v, scene.storage)


# ----------------------------------------------------------------------------------------------
# cameras and rays
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Camera:
    c2w: np.ndarray          # float32 [3, 4]: columns right, up, back, position (world)
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def packed(self) -> np.ndarray:
        """float32[18]: c2w row-major (12), fx, fy, cx, cy, then width and height bit-cast."""
        out = np.zeros(18, dtype=np.float32)
        out[:12] = self.c2w.reshape(-1)
        out[12:16] = [self.fx, self.fy, self.cx, self.cy]
        out[16:18] = np.array([self.width, self.height], dtype=np.int32).view(np.float32)
        return out

    @staticmethod
    def unpack(rec: np.ndarray) -> "Camera":
        """The camera of a packed float32[18] record (the inverse of packed())."""
        rec = np.ascontiguousarray(rec, dtype=np.float32)
        w, h = (int(x) for x in rec[16:18].view(np.int32))
        return Camera(rec[:12].reshape(3, 4).copy(), w, h, float(rec[12]), float(rec[13]),
                      float(rec[14]), float(rec[15]))


def look_at(pos, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """c2w (float32 [3,4]) of a camera at `pos` looking at `target`; x right, y up, looks down -z."""
    pos = np.asarray(pos, dtype=np.float64)
    z = pos - np.asarray(target, dtype=np.float64)
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, dtype=np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z, pos], axis=1).astype(np.float32)


def pinhole(pos, width, height, focal, target=(0.0, 0.0, 0.0)) -> Camera:
    return Camera(look_at(pos, target), int(width), int(height), float(focal), float(focal),
                  width / 2.0, height / 2.0)


def hemisphere_cameras(n: int, radius: float, width: int, height: int, focal: float,
                       seed: int) -> List[Camera]:
    """n poses on the upper (+y) hemisphere by a Fibonacci lattice with a seeded azimuth offset."""
    rng = np.random.default_rng(seed)
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    golden = np.pi * (3.0 - np.sqrt(5.0))
    cams = []
    for i in range(n):
        y = (i + 0.5) / n * 0.95
        r = math.sqrt(1.0 - y * y)
        phi = phi0 + golden * i
        pos = radius * np.array([r * math.cos(phi), y, r * math.sin(phi)])
        cams.append(pinhole(pos, width, height, focal))
    return cams


def ellipse_cameras(n: int, a: float, b: float, height_y: float, width: int, height: int,
                    focal: float, seed: int) -> List[Camera]:
    """n poses on a horizontal ellipse (semi-axes a along x, b along z) at height `height_y`."""
    rng = np.random.default_rng(seed)
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    cams = []
    for i in range(n):
        phi = phi0 + 2.0 * np.pi * i / n
        pos = np.array([a * math.cos(phi), height_y, b * math.sin(phi)])
        cams.append(pinhole(pos, width, height, focal))
    return cams


def camera_rays(cam: Camera, pixels: np.ndarray | None = None):
    """float32 rays of a pinhole camera, one per pixel in row-major order (or for `pixels`).

    Every step is one IEEE float32 operation rounded to nearest even, in this order:
      xc = ((i + 0.5) - cx) / fx ;  yc = -(((j + 0.5) - cy) / fy) ;  camera z = -1
      e_a = ((R[a,0] * xc) + (R[a,1] * yc)) - R[a,2]           for a = x, y, z
      n2 = ((e_x * e_x) + (e_y * e_y)) + (e_z * e_z) ;  inv = 1 / sqrt(n2)
      d_a = e_a * inv ;  origin = camera position
    Returns origins [n,3] and directions [n,3].
    """
    f32 = np.float32
    W, H = cam.width, cam.height
    if pixels is None:
        pixels = np.arange(W * H, dtype=np.int64)
    pixels = np.asarray(pixels, dtype=np.int64)
    i = (pixels % W).astype(np.float32)
    j = (pixels // W).astype(np.float32)
    xc = ((i + f32(0.5)) - f32(cam.cx)) / f32(cam.fx)
    yc = -(((j + f32(0.5)) - f32(cam.cy)) / f32(cam.fy))
    R = cam.c2w.astype(np.float32)
    e = [((R[a, 0] * xc) + (R[a, 1] * yc)) - R[a, 2] for a in range(3)]
    n2 = ((e[0] * e[0]) + (e[1] * e[1])) + (e[2] * e[2])
    inv = f32(1.0) / np.sqrt(n2)
    d = np.stack([e[0] * inv, e[1] * inv, e[2] * inv], axis=1).astype(np.float32)
    o = np.broadcast_to(R[:, 3], d.shape).astype(np.float32).copy()
    return np.ascontiguousarray(o), np.ascontiguousarray(d)


def ray_batch(cams: List[Camera], n_rays: int, seed: int):
    """n_rays random (view, pixel) pairs over `cams` (uniform), as float32 rays."""
    rng = np.random.default_rng(seed)
    v = rng.integers(0, len(cams), size=n_rays)
    o = np.empty((n_rays, 3), dtype=np.float32)
    d = np.empty((n_rays, 3), dtype=np.float32)
    for c in np.unique(v):
        sel = np.nonzero(v == c)[0]
        cam = cams[c]
        pix = rng.integers(0, cam.width * cam.height, size=sel.size)
        o[sel], d[sel] = camera_rays(cam, pix)
    return o, d


def random_rays(n: int, seed: int, center=(0.0, 0.0, 0.0), half=1.0, dist=3.0):
    """Rays from random points on a sphere of radius dist*half aimed at random points inside the
    root; about a tenth are exactly axis-aligned (two zero direction components)."""
    rng = np.random.default_rng(seed)
    c = np.asarray(center, dtype=np.float64)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    o = c + dist * half * u
    tgt = c + rng.uniform(-0.9 * half, 0.9 * half, size=(n, 3))
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ax = rng.random(n) < 0.1
    for r in np.nonzero(ax)[0]:
        a = int(rng.integers(0, 3))
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        o[r] = tgt[r]
        o[r, a] = c[a] - sgn * dist * half
        d[r] = 0.0
        d[r, a] = sgn
    return o.astype(np.float32), d.astype(np.float32)


# ----------------------------------------------------------------------------------------------
# the configurations of the benchmark
# ----------------------------------------------------------------------------------------------

def config_tiny():
    """64x64 camera at distance 3 (focal 80) on the tiny sphere scene; white background."""
    sc = tiny_sphere_scene(seed=0)
    cams = [pinhole((0.0, 0.0, 3.0), 64, 64, 80.0)]
    return sc, cams


def config_nerf_synthetic(n_views: int = 100):
    """100 views of 800x800 on a radius-4 hemisphere, focal 1111, on the NeRF-synthetic-shaped scene."""
    sc = nerf_synthetic_scene(seed=1000)
    cams = hemisphere_cameras(n_views, 4.0, 800, 800, 1111.0, seed=1001)
    return sc, cams


def config_tanks_temples(n_views: int = 150):
    """150 views of 1920x1080 on an ellipse (5.0 / 4.5, height 1.5), focal 1200."""
    sc = tanks_temples_scene(seed=3000)
    cams = ellipse_cameras(n_views, 5.0, 4.5, 1.5, 1920, 1080, 1200.0, seed=3001)
    return sc, cams


def config_train(n_views: int = 100):
    """The differentiable-training configuration: the tiny sphere scene (depth 4, FP32, SH degree
    1) and 100 views of 800x800 on a radius-3 upper hemisphere, focal 1000 (the field of view of
    the tiny scene's own 64x64, focal-80 camera at distance 3)."""
    sc = tiny_sphere_scene(seed=0)
    cams = hemisphere_cameras(n_views, 3.0, 800, 800, 1000.0, seed=2001)
    return sc, cams


def perturbed_params(sigma: np.ndarray, sh: np.ndarray, seed: int):
    """The seeded perturbed copy of a tree's leaf parameters that training targets are rendered
    from: every density times U(0.8, 1.2), every SH coefficient plus N(0, 0.1), in float32 (one
    rounding each), leaf by leaf in the given order."""
    rng = np.random.default_rng(seed)
    s = np.asarray(sigma, np.float32) * rng.uniform(0.8, 1.2, size=np.shape(sigma)).astype(np.float32)
    h = np.asarray(sh, np.float32) + rng.normal(0.0, 0.1, size=np.shape(sh)).astype(np.float32)
    return s.astype(np.float32), h.astype(np.float32)


def random_signal(n: int, seed: int, tie_fraction: float = 0.2) -> np.ndarray:
    """Non-negative float32 signal with many exact ties (a fifth of the values repeat)."""
    rng = np.random.default_rng(seed)
    s = rng.exponential(1.0, size=n).astype(np.float32)
    k = int(n * tie_fraction)
    if k and n > 1:
        idx = rng.integers(0, n, size=k)
        s[idx] = s[rng.integers(0, n, size=k)]
        s[rng.integers(0, n, size=max(1, k // 4))] = 0.0
    return s


def signed_signal(n: int, seed: int, p_pos: float = 0.3, p_zero: float = 0.4,
                  p_nan: float = 0.05) -> np.ndarray:
    """Float32 signal of positive values (a fifth of them repeated), +0.0 and -0.0 in equal
    shares, negative values and NaNs, in random leaf order: a per-leaf signal such as raw
    densities can hold all of these."""
    rng = np.random.default_rng(seed)
    u = rng.random(n)
    s = -rng.exponential(1.0, size=n).astype(np.float32)
    pos = u < p_pos
    s[pos] = rng.exponential(1.0, size=int(pos.sum())).astype(np.float32)
    idx = np.flatnonzero(pos)
    if idx.size > 1:
        k = idx.size // 5
        s[rng.choice(idx, k)] = s[rng.choice(idx, k)]
    zero = (u >= p_pos) & (u < p_pos + p_zero)
    s[zero] = np.where(rng.random(int(zero.sum())) < 0.5, np.float32(-0.0), np.float32(0.0))
    s[u >= 1.0 - p_nan] = np.nan
    return s


def random_masks(n: int, seed: int, p_prune: float = 0.6, p_sample: float = 0.05):
    rng = np.random.default_rng(seed)
    prune = (rng.random(n) < p_prune).astype(np.uint8)
    sample = (rng.random(n) < p_sample).astype(np.uint8)
    return prune, sample


# ----------------------------------------------------------------------------------------------
# serving workload
# ----------------------------------------------------------------------------------------------

SERVE_RESOLUTIONS = [(256, 256), (512, 512), (800, 800), (1280, 720), (1920, 1080)]


def config_serving():
    """Four resident scenes for the serving loop: the tiny sphere scene (FP32, SH degree 1), the
    same scene again as the tree the training configuration leaves after its refines (the caller
    refines it: the benchmark serves the tree its training run produced, the tests refine it with
    seeded marks), and two seed variants of the NeRF-synthetic-shaped scene (FP16, SH degree 3).
    Also a pose sampler: a random direction on the upper hemisphere at the scene's viewing
    distance, focal scaled with the width as in the scene's own camera (80 per 64 px for the
    tiny scene, 1111 per 800 px for the NeRF-synthetic-shaped one)."""
    scenes = [tiny_sphere_scene(seed=0), tiny_sphere_scene(seed=0),
              nerf_synthetic_scene(seed=1010), nerf_synthetic_scene(seed=1020)]
    refined = [False, True, False, False]
    dist = [3.0, 3.0, 4.0, 4.0]
    focal_per_px = [80.0 / 64.0, 80.0 / 64.0, 1111.0 / 800.0, 1111.0 / 800.0]

    def poses(rng, tree, w, h):
        y = rng.uniform(0.05, 0.95)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        r = math.sqrt(1.0 - y * y)
        pos = dist[tree] * np.array([r * math.cos(phi), y, r * math.sin(phi)])
        return pinhole(pos, w, h, focal_per_px[tree] * w).packed()

    return scenes, refined, poses
