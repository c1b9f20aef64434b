"""Checks of the seeded input generators (no GPU)."""
import numpy as np
import pytest

import seeded_inputs as si


def test_splitmix64_reference_sequence():
    # first outputs of SplitMix64 seeded with 1234567 (the reference C implementation's sequence)
    out = si.splitmix64(1234567, np.arange(5, dtype=np.uint64)).tolist()
    assert out == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 10000), rng.normal(0, 1e-30, 100)]).astype(np.float32)
    ours = si.f32_to_bf16_bits(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)


def test_leaf_param_moments():
    sc = si.nerf_synthetic_scene()
    keys = np.arange(1 << 27, (1 << 27) + 20000, dtype=np.uint64)
    inside = np.ones(keys.size, bool)
    inside[::3] = False
    sig, sh = si.leaf_params(keys, inside, sc)
    s = sig.astype(np.float64)
    assert np.all(s[~inside] == 0)
    assert s[inside].min() >= 10 and s[inside].max() <= 200
    assert abs(s[inside].mean() - 105) < 3
    v = sh.astype(np.float64)
    assert abs(v[:, :, 1:].std() - 0.5) < 0.01
    assert abs(v[:, :, 0].mean() - 0.5) < 0.01
    # keyed by the leaf key: the same key gives the same draw regardless of position
    sig2, sh2 = si.leaf_params(keys[::-1], inside[::-1], sc)
    np.testing.assert_array_equal(sig2[::-1], sig)
    np.testing.assert_array_equal(sh2[::-1], sh)


def test_camera_rays_unit_and_centred():
    cam = si.pinhole((0.0, 0.0, 3.0), 64, 64, 80.0)
    o, d = si.camera_rays(cam)
    assert o.shape == (4096, 3) and d.dtype == np.float32
    np.testing.assert_allclose(np.linalg.norm(d.astype(np.float64), axis=1), 1.0, atol=1e-6)
    # the four pixels around the image centre point symmetrically about -z
    c = d.reshape(64, 64, 3)[31:33, 31:33]
    assert np.all(c[..., 2] < -0.9999)
    np.testing.assert_array_equal(np.abs(c[0, 0]), np.abs(c[1, 1]))


def test_config_shapes():
    sc, cams = si.config_nerf_synthetic()
    assert len(cams) == 100 and cams[0].width == 800 and sc.max_depth == 9
    sc, cams = si.config_tanks_temples()
    assert len(cams) == 150 and cams[0].width == 1920 and cams[0].height == 1080
    for c in cams:
        assert abs(np.linalg.norm(c.c2w[:, 3]) - 0) > 4.4
