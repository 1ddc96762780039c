"""Pins of the FP64 reference network: the hand-written backward pass
against central finite differences of the loss, and one Adam step against
its closed form on a quadratic."""
import numpy as np

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = mlp.init_params(seed=1) + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = rng.uniform(-1, 1, (40, 2))
    t = rng.normal(0, 1, 40)
    _, g = mlp.loss_and_grad(w, x, t)
    idx = rng.choice(mlp.N_PARAMS, 80, replace=False)
    idx = np.r_[idx, [0, 127, 128, 191, mlp.N_PARAMS - 65, mlp.N_PARAMS - 1]]
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, x, t)[0] - mlp.loss_and_grad(wm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_silu_derivative():
    a = np.linspace(-8, 8, 101)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(a), (mlp.silu(a + h) - mlp.silu(a - h)) / (2 * h), atol=1e-8)


def test_adam_first_step_moves_by_lr():
    # bias correction makes the first step -lr * sign(g) (for |g| >> eps)
    w = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    w2, m, v = mlp.adam_step(w, g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(w2, w - 0.01 * np.sign(g), rtol=1e-6)
