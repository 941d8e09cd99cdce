"""The float64 reference network against central finite differences."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    n_in, h, B = 7, 9, 13
    P = h * n_in + h + h * h + h + h + 1
    theta = rng.normal(0, 0.5, P)
    X = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, B)
    g = mlp.gradients(theta, X, t, n_in, h)
    eps = 1e-6
    for i in rng.choice(P, 60, replace=False):
        tp = theta.copy(); tp[i] += eps
        tm = theta.copy(); tm[i] -= eps
        fd = (mlp.loss(tp, X, t, n_in, h) - mlp.loss(tm, X, t, n_in, h)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd)


def test_adamw_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    th, m, v = mlp.adamw_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.0)
    # bias-corrected first step moves each weight by lr * sign(g) (eps aside)
    assert np.allclose(th[:2], theta[:2] - 0.01 * np.sign(g[:2]), atol=1e-9)
    assert th[2] == theta[2]
    th2, _, _ = mlp.adamw_step(theta, np.zeros(3), np.zeros(3), np.zeros(3), 1, lr=0.01, wd=0.1)
    assert np.allclose(th2, theta * (1 - 0.001))


def test_adamw_constant_gradient_moves_lr_per_step():
    # with a constant gradient g the bias-corrected moments are exactly g and
    # g^2 at every step t (m_t = (1 - b1^t) g, v_t = (1 - b2^t) g^2), so each
    # step moves a weight by lr * g / (|g| + eps); a wrong bias correction
    # (1 - b^step) shows up from step 2 on
    theta = np.array([1.0, -2.0, 0.5, 3.0])
    g = np.array([0.3, -0.1, 2.0, -7.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    for step in range(1, 8):
        th, m, v = mlp.adamw_step(theta, g, m, v, step, lr=lr, wd=0.0, eps=eps)
        np.testing.assert_allclose(th - theta, -lr * g / (np.abs(g) + eps), rtol=1e-10, atol=1e-15)
        theta = th


def test_adamw_second_step_closed_form():
    # g1 = g, g2 = -g: m_hat_2 = (b1 g1 + g2) / (1 + b1) = -g / 19 and
    # v_hat_2 = (b2 g1^2 + g2^2) / (1 + b2) = g^2, so step 2 moves by
    # +lr * sign(g) / 19 (eps aside); with weight decay wd the decoupled term
    # -lr * wd * theta is added
    theta0 = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 4.0])
    lr, wd = 0.02, 0.05
    th1, m, v = mlp.adamw_step(theta0, g, np.zeros(3), np.zeros(3), 1, lr=lr, wd=wd)
    th2, m, v = mlp.adamw_step(th1, -g, m, v, 2, lr=lr, wd=wd)
    want = th1 - lr * (-(g / 19.0) / (np.abs(g) + 1e-8) + wd * th1)
    np.testing.assert_allclose(th2, want, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m, -0.01 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001999 * g * g, rtol=1e-12)


def test_rounded_layer2_gradient_only_changes_the_two_products():
    # rnd_dz stores the layer-2 pre-activation gradient in a coarser format
    # only where it enters the W2 gradient and the gradient passed to layer 1:
    # every other block (W3, b3, b2) is unchanged, and with an identity
    # rounding nothing changes
    rng = np.random.default_rng(3)
    n_in, h, B = 5, 8, 11
    P = h * n_in + h + h * h + h + h + 1
    theta = rng.normal(0, 0.5, P)
    X = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, B)
    g = mlp.gradients(theta, X, t, n_in, h)
    assert np.array_equal(g, mlp.gradients(theta, X, t, n_in, h, rnd_dz=lambda a: a))
    coarse = mlp.gradients(theta, X, t, n_in, h, rnd_dz=lambda a: np.round(a * 8) / 8)
    o_w2 = h * n_in + h
    o_b2 = o_w2 + h * h
    assert np.array_equal(g[o_b2:], coarse[o_b2:])
    assert not np.array_equal(g[o_w2:o_b2], coarse[o_w2:o_b2])
    assert not np.array_equal(g[:h * n_in], coarse[:h * n_in])
