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
