"""Pins of the oracle's optimisation step (no GPU): the MSE loss of Algorithm 1 (optimization)
and the RMSProp update of Sec. 3.3, fixed against closed forms, PyTorch's RMSprop in float64,
finite differences, and the end-to-end chain MSE(render(params)) by finite differences."""

import numpy as np
import pytest

import oracle
import seeded_inputs as si


def test_mse_small_case_by_hand():
    rgb = np.array([[0.5, 0.25, 1.0], [0.0, 0.0, 0.0]])
    tgt = np.array([[0.0, 0.25, 0.5], [1.0, 0.0, 0.0]])
    loss, g = oracle.mse(rgb, tgt)
    # squared errors 0.25, 0, 0.25, 1, 0, 0 over 6 entries
    assert loss == pytest.approx(1.5 / 6, abs=1e-15)
    np.testing.assert_allclose(g, 2 * (rgb - tgt) / 6, atol=1e-15)


def test_mse_gradient_by_finite_differences():
    rng = np.random.default_rng(3)
    rgb, tgt = rng.random((7, 3)), rng.random((7, 3))
    _, g = oracle.mse(rgb, tgt)
    h = 1e-6
    for i in range(7):
        for c in range(3):
            a, b = rgb.copy(), rgb.copy()
            a[i, c] += h
            b[i, c] -= h
            fd = (oracle.mse(a, tgt)[0] - oracle.mse(b, tgt)[0]) / (2 * h)
            assert fd == pytest.approx(g[i, c], rel=1e-7, abs=1e-10)


def test_rmsprop_constant_gradient_closed_form():
    """A constant gradient g from ms = 0: ms_n = (1 - rho^n) g^2 and, with eps = 0,
    p_n = p_0 - lr sign(g) sum_k (1 - rho^k)^(-1/2)."""
    rho, lr = 0.9, 0.05
    g = np.array([0.3, -2.0, 1e-3])
    p, ms = np.array([1.0, -1.0, 0.5]), np.zeros(3)
    p0 = p.copy()
    for n in range(1, 13):
        p, ms = oracle.rmsprop(p, ms, g, lr, rho, 0.0)
        np.testing.assert_allclose(ms, (1 - rho ** n) * g * g, rtol=1e-14)
        steps = sum((1 - rho ** k) ** -0.5 for k in range(1, n + 1))
        np.testing.assert_allclose(p, p0 - lr * np.sign(g) * steps, rtol=1e-13)


def test_rmsprop_scale_invariance_without_eps():
    rng = np.random.default_rng(4)
    p, ms, g = rng.normal(size=50), rng.random(50), rng.normal(size=50)
    a, _ = oracle.rmsprop(p, ms, g, 0.1, 0.95, 0.0)
    b, _ = oracle.rmsprop(p, ms * 49.0, g * 7.0, 0.1, 0.95, 0.0)
    np.testing.assert_allclose(a, b, rtol=1e-14)


def test_rmsprop_matches_torch_rmsprop():
    """torch.optim.RMSprop (alpha = rho, no momentum, not centred) in float64."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=64)
    grads = [rng.normal(size=64) * s for s in (1.0, 0.1, 3.0, 0.5)]
    w = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.RMSprop([w], lr=0.01, alpha=0.9, eps=1e-8)
    p, ms = p0.copy(), np.zeros(64)
    for g in grads:
        opt.zero_grad()
        w.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, ms = oracle.rmsprop(p, ms, g, 0.01, 0.9, 1e-8)
    np.testing.assert_allclose(p, w.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_training_gradient_chain_by_finite_differences():
    """d MSE(render(sigma, sh), target) / d params by central differences of the oracle's render
    and loss, against backward(grad of the loss) -- the chain one training step takes."""
    sc = si.random_scene(31, max_depth=3, sh_degree=1, n_prims=2)
    t = oracle.scene_tree(sc)
    lo, size = oracle.root_of(sc)
    L, K = t["leaf_key"].size, 4
    rng = np.random.default_rng(6)
    sigma = rng.uniform(0.5, 3.0, L)
    sh = rng.normal(0, 0.4, (L, 3, K))
    o, d = si.random_rays(30, 11)
    tgt = rng.random((30, 3))

    def loss(sg, shh):
        rgb, _, _ = oracle.render(t, lo, size, sg, shh, 1, o, d, eps_T=0.0)
        return oracle.mse(rgb, tgt)[0]

    rgb, _, _ = oracle.render(t, lo, size, sigma, sh, 1, o, d, eps_T=0.0)
    _, g = oracle.mse(rgb, tgt)
    gs, gsh, _, _ = oracle.backward(t, lo, size, sigma, sh, 1, o, d, g, eps_T=0.0)
    h = 1e-6
    touched = np.nonzero(np.abs(gs) > 0)[0]
    assert touched.size >= 3
    for v in touched[:8]:
        a, b = sigma.copy(), sigma.copy()
        a[v] += h
        b[v] -= h
        assert (loss(a, sh) - loss(b, sh)) / (2 * h) == pytest.approx(gs[v], rel=1e-5, abs=1e-9)
        for ch, k in ((0, 0), (2, 3)):
            a, b = sh.copy(), sh.copy()
            a[v, ch, k] += h
            b[v, ch, k] -= h
            fd = (loss(sigma, a) - loss(sigma, b)) / (2 * h)
            assert fd == pytest.approx(gsh[v, ch, k], rel=1e-5, abs=1e-9)
