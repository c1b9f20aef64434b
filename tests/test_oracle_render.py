"""Pins of the oracle's segments, SH, volume rendering (Eq. 1-2), gradients and signal (no GPU).

Each check fixes the oracle to something other than itself: quadrature, scipy's spherical
harmonics, closed forms for constant density, brute-force fine-step marching, finite
differences, and refinement invariants.
"""
import math

import numpy as np
import pytest

import oracle
import seeded_inputs as si

# ----------------------------------------------------------------------------------------------
# spherical harmonics
# ----------------------------------------------------------------------------------------------


def _quadrature():
    """Gauss-Legendre (8 nodes) in cos(theta) x 16 uniform phi: exact for degree <= 7."""
    x, w = np.polynomial.legendre.leggauss(8)
    phi = (np.arange(16) + 0.5) * 2 * np.pi / 16
    dirs, wts = [], []
    for xi, wi in zip(x, w):
        s = math.sqrt(1 - xi * xi)
        for p in phi:
            dirs.append((s * math.cos(p), s * math.sin(p), xi))
            wts.append(wi * 2 * np.pi / 16)
    return np.array(dirs), np.array(wts)


def test_sh_orthonormal_by_quadrature():
    dirs, wts = _quadrature()
    Y = np.stack([oracle.sh_basis(3, d) for d in dirs])       # [n, 16]
    G = (Y * wts[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-13


def test_sh_dc_constant():
    assert oracle.sh_basis(0, [0.0, 0.0, 1.0])[0] == pytest.approx(1 / (2 * math.sqrt(math.pi)), abs=1e-16)


def test_sh_matches_scipy_up_to_sign():
    """Each basis function equals +-1 x scipy's real spherical harmonic of the same (l, m), with
    the sign fixed per function; z is the polar axis, m < 0 the sine (y) family."""
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(0)
    d = rng.normal(size=(64, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    ours = np.stack([oracle.sh_basis(3, x) for x in d])
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            Yc = sp.sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                ref = Yc.real
            elif m > 0:
                ref = math.sqrt(2) * Yc.real
            else:
                ref = math.sqrt(2) * Yc.imag
            s = np.sign(np.dot(ours[:, k], ref))
            assert s != 0
            np.testing.assert_allclose(ours[:, k], s * ref, atol=1e-13)


def test_sh_addition_theorem():
    """sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.normal(size=(2, 3))
        a /= np.linalg.norm(a)
        b /= np.linalg.norm(b)
        Ya, Yb = oracle.sh_basis(3, a), oracle.sh_basis(3, b)
        for l in range(4):
            sl = slice(l * l, (l + 1) ** 2)
            lhs = float(np.dot(Ya[sl], Yb[sl]))
            P = np.polynomial.legendre.legval(float(np.dot(a, b)), [0] * l + [1])
            assert lhs == pytest.approx((2 * l + 1) / (4 * np.pi) * P, abs=1e-13)


# ----------------------------------------------------------------------------------------------
# segments
# ----------------------------------------------------------------------------------------------

def _full_tree(D, half=1.0):
    """A box covering the whole root: every cell is subdivided down to depth D."""
    sc = si.box_scene((-2 * half,) * 3, (2 * half,) * 3, half=half, max_depth=D)
    return sc, oracle.scene_tree(sc)


def test_segments_axis_aligned_full_tree():
    sc, t = _full_tree(3)
    lo, size = oracle.root_of(sc)
    cell = size / 8
    for a in range(3):
        for sgn in (1.0, -1.0):
            o = np.array([-0.875 + 0.25 * 2, 0.125, -0.375], np.float32)  # cell centres
            d = np.zeros(3, np.float32)
            d[a] = sgn
            o[a] = -3.0 * sgn
            leaf, ti, to = oracle.segments(t, lo, size, o, d)
            assert len(leaf) == 8
            np.testing.assert_array_equal(to - ti, np.full(8, cell))
            assert len(set(leaf.tolist())) == 8


@pytest.mark.parametrize("seed", [0, 1])
def test_segments_tile_the_root_chord(seed):
    sc = si.random_scene(seed, max_depth=5, n_prims=4)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    o, d = si.random_rays(300, seed + 10)
    for r in range(300):
        leaf, ti, to = oracle.segments(t, lo, size, o[r], d[r])
        if len(leaf) == 0:
            continue
        # contiguous and increasing
        np.testing.assert_allclose(ti[1:], to[:-1], rtol=0, atol=1e-12)
        assert np.all(to > ti)
        # total = root chord (slab test written out here)
        oo = (o[r].astype(np.float64) - lo) / size
        dd = d[r].astype(np.float64) / size
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = np.where(dd != 0, (0 - oo) / dd, -np.inf)
            t1 = np.where(dd != 0, (1 - oo) / dd, np.inf)
        tn = max(0.0, np.max(np.minimum(t0, t1)))
        tf = np.min(np.maximum(t0, t1))
        assert (to - ti).sum() == pytest.approx(tf - tn, abs=1e-12)


# ----------------------------------------------------------------------------------------------
# rendering: closed forms and brute force
# ----------------------------------------------------------------------------------------------

C0 = 1 / (2 * math.sqrt(math.pi))


def test_constant_density_cube_closed_form():
    """All leaves of one density s, DC-only linear colour c: C = (1 - e^{-sL}) c + e^{-sL} bg."""
    sc, t = _full_tree(3)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    s, c = 1.7, np.array([0.2, 0.5, 0.9])
    sigma = np.full(L, s)
    sh = np.zeros((L, 3, 1))
    sh[:, :, 0] = c / C0
    bg = np.array([1.0, 0.25, 0.0])
    o, d = si.random_rays(500, 3)
    rgb, T, _ = oracle.render(t, lo, size, sigma, sh, 0, o, d, bg=bg, eps_T=0.0,
                              color_act=oracle.ACT_LINEAR)
    for r in range(500):
        oo = (o[r].astype(np.float64) - lo) / size
        dd = d[r].astype(np.float64) / size
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = np.where(dd != 0, -oo / dd, -np.inf)
            t1 = np.where(dd != 0, (1 - oo) / dd, np.inf)
        tn, tf = max(0.0, np.max(np.minimum(t0, t1))), np.min(np.maximum(t0, t1))
        chord = max(0.0, tf - tn)
        Te = math.exp(-s * chord)
        assert T[r] == pytest.approx(Te, rel=1e-12, abs=1e-15)
        np.testing.assert_allclose(rgb[r], (1 - Te) * c + Te * bg, rtol=1e-12, atol=1e-14)


def _march(tree, lo, size, sigma, sh, o, d, h, bg):
    """Brute-force midpoint marching with step h (DC-only linear colour), independent of the
    oracle's segment code: point location by descending child pointers."""
    oo = (o.astype(np.float64) - lo) / size
    dd = d.astype(np.float64) / size
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = np.where(dd != 0, -oo / dd, -np.inf)
        t1 = np.where(dd != 0, (1 - oo) / dd, np.inf)
    tn, tf = max(0.0, np.max(np.minimum(t0, t1))), np.min(np.maximum(t0, t1))
    T, C = 1.0, np.zeros(3)
    if not tf > tn:
        return C + bg
    n = int(math.ceil((tf - tn) / h))
    hh = (tf - tn) / n
    for i in range(n):
        p = oo + (tn + (i + 0.5) * hh) * dd
        node, l = 0, 0
        while True:
            b = np.minimum((p * (1 << (l + 1))).astype(np.int64), (1 << (l + 1)) - 1) & 1
            ch = tree["child"][node, 4 * b[0] + 2 * b[1] + b[2]]
            l += 1
            if ch < 0:
                v = -1 - ch
                break
            node = ch
        a = 1 - math.exp(-max(sigma[v], 0) * hh)
        C += T * a * sh[v, :, 0] * C0
        T *= 1 - a
    return C + T * bg


def test_bruteforce_marching_converges():
    sc = si.random_scene(11, max_depth=3, sh_degree=0, n_prims=3)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(5)
    sigma = rng.uniform(0.0, 3.0, L)
    sigma[rng.random(L) < 0.3] = 0.0
    sh = rng.uniform(0, 2, (L, 3, 1))
    bg = np.array([1.0, 1.0, 1.0])
    o, d = si.random_rays(12, 8)
    rgb, _, _ = oracle.render(t, lo, size, sigma, sh, 0, o, d, bg=bg, eps_T=0.0,
                              color_act=oracle.ACT_LINEAR)
    for r in range(12):
        e1 = np.abs(_march(t, lo, size, sigma, sh, o[r], d[r], 2e-3, bg) - rgb[r]).max()
        e2 = np.abs(_march(t, lo, size, sigma, sh, o[r], d[r], 2e-4, bg) - rgb[r]).max()
        assert e2 < 2e-3           # O(sigma_max h) with cell-boundary samples straddling
        assert e2 <= e1 + 1e-12


def test_early_termination_stops_after_threshold():
    sc, t = _full_tree(3)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    sigma = np.full(L, 40.0)
    sh = np.zeros((L, 3, 1))
    o, d = si.random_rays(50, 4)
    rgb, T, nseg = oracle.render(t, lo, size, sigma, sh, 0, o, d, eps_T=1e-4)
    _, T0, nseg0 = oracle.render(t, lo, size, sigma, sh, 0, o, d, eps_T=0.0)
    for r in range(50):
        leaf, ti, to = oracle.segments(t, lo, size, o[r], d[r])
        Tc = np.exp(-40.0 * np.cumsum(to - ti))
        below = np.nonzero(Tc < 1e-4)[0]
        expect = below[0] + 1 if below.size else len(leaf)
        assert nseg[r] == expect and nseg0[r] == len(leaf)
        assert T[r] == pytest.approx(Tc[expect - 1] if expect else 1.0, rel=1e-12)


# ----------------------------------------------------------------------------------------------
# gradients
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("act", [oracle.ACT_SIGMOID, oracle.ACT_LINEAR])
def test_gradient_finite_differences(act):
    sc = si.random_scene(21, max_depth=3, sh_degree=2, n_prims=3)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    L, K = t["leaf_key"].size, 9
    rng = np.random.default_rng(2)
    sigma = rng.uniform(0.5, 4.0, L)
    sigma[rng.random(L) < 0.2] = -1.0              # inactive (ReLU) leaves
    sh = rng.normal(0, 0.5, (L, 3, K))
    o, d = si.random_rays(40, 9)
    g = rng.normal(size=(40, 3))
    bg = (0.3, 0.6, 0.9)

    def loss(sg, shh):
        rgb, _, _ = oracle.render(t, lo, size, sg, shh, 2, o, d, bg=bg, eps_T=0.0, color_act=act)
        return float((rgb * g).sum())

    gs, gsh, _, _ = oracle.backward(t, lo, size, sigma, sh, 2, o, d, g, bg=bg, eps_T=0.0,
                                    color_act=act)
    h = 1e-6
    touched = np.nonzero(np.abs(gs) > 0)[0]
    assert touched.size > 5
    for v in touched[:25]:
        sp, sm = sigma.copy(), sigma.copy()
        sp[v] += h
        sm[v] -= h
        fd = (loss(sp, sh) - loss(sm, sh)) / (2 * h)
        assert gs[v] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert np.all(gs[sigma <= 0] == 0)
    flat = np.argwhere(np.abs(gsh) > 1e-6)
    for (v, ch, k) in flat[rng.permutation(len(flat))[:25]]:
        sp, sm = sh.copy(), sh.copy()
        sp[v, ch, k] += h
        sm[v, ch, k] -= h
        fd = (loss(sigma, sp) - loss(sigma, sm)) / (2 * h)
        assert gsh[v, ch, k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_gradient_with_early_termination_matches_fd():
    """With eps_T > 0 the render is a fixed truncation away from the stopping segment; its
    derivative is the truncated sum (checked by differences that do not move the stop)."""
    sc, t = _full_tree(3)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    rng = np.random.default_rng(3)
    sigma = rng.uniform(5, 30, L)
    sh = rng.normal(0, 0.5, (L, 3, 4))
    o, d = si.random_rays(20, 12)
    g = rng.normal(size=(20, 3))

    def loss(sg):
        rgb, _, _ = oracle.render(t, lo, size, sg, sh, 1, o, d, eps_T=1e-3)
        return float((rgb * g).sum())

    gs, _, _, _ = oracle.backward(t, lo, size, sigma, sh, 1, o, d, g, eps_T=1e-3)
    _, _, n1 = oracle.render(t, lo, size, sigma, sh, 1, o, d, eps_T=1e-3)
    h = 1e-7
    for v in np.nonzero(gs)[0][:20]:
        sp, sm = sigma.copy(), sigma.copy()
        sp[v] += h
        sm[v] -= h
        _, _, n2 = oracle.render(t, lo, size, sp, sh, 1, o, d, eps_T=1e-3)
        _, _, n3 = oracle.render(t, lo, size, sm, sh, 1, o, d, eps_T=1e-3)
        if not (np.array_equal(n1, n2) and np.array_equal(n1, n3)):
            continue
        fd = (loss(sp) - loss(sm)) / (2 * h)
        assert gs[v] == pytest.approx(fd, rel=1e-5, abs=1e-8)


# ----------------------------------------------------------------------------------------------
# signal (Sec. 3.1)
# ----------------------------------------------------------------------------------------------

def test_signal_closed_form_axis_rays():
    """Axis-aligned rays through cell centres of a full depth-2 constant-density tree: every leaf
    on a ray gets alpha = 1 - exp(-s cell); the i-th leaf's weight is e^{-s cell i} alpha."""
    sc, t = _full_tree(2)
    lo, size = oracle.root_of(sc)
    L = t["leaf_key"].size
    s = 0.8
    sigma = np.full(L, s)
    sh = np.zeros((L, 3, 1))
    cell = size / 4
    centres = -1 + 0.25 + 0.5 * np.arange(4)
    o, d = [], []
    for x in centres:
        for y in centres:
            o.append((x, y, 3.0))
            d.append((0, 0, -1.0))
    o, d = np.array(o, np.float32), np.array(d, np.float32)
    S = np.zeros(L)
    oracle.render(t, lo, size, sigma, sh, 0, o, d, eps_T=0.0, signal=S,
                  signal_mode=oracle.SIGNAL_SUM_ALPHA)
    np.testing.assert_allclose(S, np.full(L, 1 - math.exp(-s * cell)), rtol=1e-13)
    W = np.zeros(L)
    oracle.render(t, lo, size, sigma, sh, 0, o, d, eps_T=0.0, signal=W,
                  signal_mode=oracle.SIGNAL_MAX_WEIGHT)
    a = 1 - math.exp(-s * cell)
    # the leaf at depth index i along -z (z from high to low) has weight e^{-s cell i} a
    for v, key in enumerate(t["leaf_key"]):
        kz = int(key) & 1 | ((int(key) >> 3) & 1) << 1
        i = 3 - kz
        assert W[v] == pytest.approx(math.exp(-s * cell * i) * a, rel=1e-13)
