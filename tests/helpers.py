"""Shared helpers of the parity tests: oracle-side trees and parameters, GPU-side trees, and the
tolerances the comparisons use."""
import numpy as np

import oracle
import seeded_inputs as si

# FP32 leaves, exact mode: |gpu - oracle| <= REL * max(|oracle|, FLOOR) per channel; a ray may
# exceed it only when it grazes a cell edge or corner within float32 resolution (at most 0.1% of
# rays, and never by more than GRAZE).
REL = 1e-5
FLOOR = 1e-2
GRAZE = 1e-3
# 16-bit leaves, fast mode: absolute per channel
ABS16 = 2e-3


def oracle_side(scene):
    """The oracle's own tree and the seeded parameters of its leaves (float64 copies)."""
    t = oracle.scene_tree(scene)
    sig, sh = si.leaf_params(t["leaf_key"], t["leaf_inside"], scene)
    return t, sig, sh, si.storage_to_f64(sig, scene.storage), si.storage_to_f64(sh, scene.storage)


def assert_pixels_close(got, ref, storage, exact=True, what="rgb"):
    got = np.asarray(got, np.float64).reshape(ref.shape)
    if storage == si.STORAGE_F32 and exact:
        err = np.abs(got - ref) / np.maximum(np.abs(ref), FLOOR)
        bad = err > REL
        if ref.ndim > 1:
            bad = bad.reshape(ref.shape[0], -1).any(axis=1)
        assert bad.mean() <= 1e-3, f"{what}: {bad.sum()} of {bad.size} rays beyond {REL} (max {err.max():.3g})"
        assert err.max() <= GRAZE, f"{what}: max relative error {err.max():.3g}"
        return err
    err = np.abs(got - ref)
    assert err.max() <= ABS16, f"{what}: max abs error {err.max():.3g}"
    return err


def assert_sums_close(got, ref, absum, rel, what="grad", floor=1e-7):
    """A float32 sum of many terms against the FP64 sum: |d| <= rel * sum|terms| + floor."""
    got = np.asarray(got, np.float64).reshape(ref.shape)
    d = np.abs(got - ref)
    lim = rel * absum + floor
    bad = d > lim
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} beyond tolerance; worst excess "
                           f"{(d - lim).max():.3g} at |ref| {np.abs(ref).flat[np.argmax(d - lim)]:.3g}")


def bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint8)


def assert_sums_close_grazing(got, ref, absum, rel, what, floor, max_leaf_frac=1e-3, cap_abs=None):
    """assert_sums_close for the sums of a large ray batch in fast mode: a ray that grazes a cell
    face moves the ends of a sliver segment by ~1e-7 of the root over |d_a|, which is unbounded
    relative to the sliver's own tiny weight, so a leaf whose sum holds few terms can exceed
    `rel`.  At most max_leaf_frac of the leaves with any gradient may, and none by more than
    cap_abs in absolute terms (default 100 x floor).  Returns (leaves beyond rel, leaves with a
    gradient, worst absolute excess over rel * sum|terms| in units of floor)."""
    got = np.asarray(got, np.float64).reshape(ref.shape)
    d = np.abs(got - ref)
    lead = ref.shape[0]
    cap_abs = 100 * floor if cap_abs is None else cap_abs
    bad = (d > rel * absum + floor).reshape(lead, -1).any(axis=1)
    live = (absum > 0).reshape(lead, -1).any(axis=1)
    worst = float(np.max(d - rel * absum, initial=0.0) / floor)
    n_bad, n_live = int(bad.sum()), int(live.sum())
    assert n_bad <= max_leaf_frac * n_live, f"{what}: {n_bad} of {n_live} leaves beyond {rel}"
    assert not (d > rel * absum + cap_abs).any(), f"{what}: worst excess {worst:.3g} x floor"
    return n_bad, n_live, worst
