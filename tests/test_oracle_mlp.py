"""Pins of the surrogate network's oracle: analytic gradients against central
finite differences (FP64), GELU against its defining formula's limits and
derivative, AdamW's first step against its closed form."""
import math

import numpy as np

from oracle import mlp


def _tiny(seed=0, n=7, n_coef=40):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(mlp.param_count(n_coef)) * 0.2
    feat = rng.standard_normal((n, mlp.FEAT)) * 0.5
    coef = rng.standard_normal((n, n_coef)) * 0.3
    target = rng.standard_normal(n)
    return flat, feat, coef, target


def test_gradients_match_finite_differences():
    n_coef = 40
    flat, feat, coef, target = _tiny(n_coef=n_coef)
    p = mlp.unpack(flat, n_coef)
    loss, g = mlp.loss_and_grads(p, feat, coef, target)
    gflat = mlp.pack(g, n_coef)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(flat), 60, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unpack(fp, n_coef), feat, coef, target)
        lm, _ = mlp.loss_and_grads(mlp.unpack(fm, n_coef), feat, coef, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_gelu_limits_and_derivative():
    z = np.array([-30.0, -3.0, -0.5, 0.0, 0.5, 3.0, 30.0])
    y = mlp.gelu(z)
    assert y[3] == 0.0 and abs(y[0]) < 1e-12 and abs(y[-1] - 30.0) < 1e-12
    # gelu(z) - gelu(-z) = z exactly for the tanh form (odd tanh)
    assert np.allclose(mlp.gelu(z) - mlp.gelu(-z), z, atol=1e-15)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(fd, mlp.gelu_grad(z), atol=1e-8)
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5


def test_adamw_first_step_closed_form():
    # at step 1 the bias-corrected moments are g and g^2: the update is
    # lr * (g / (|g| + eps) + wd p)
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    newp, m, v = mlp.adamw(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=1e-8, wd=0.1)
    want = p - 0.01 * (g / (np.abs(g) + 1e-8) + 0.1 * p)
    assert np.allclose(newp, want, rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_parameter_layout():
    assert mlp.param_count(320) == 64 * 320 + 256 * 80 + 256 + 2 * (256 * 256 + 256) + 256 + 1
    flat = np.arange(mlp.param_count(40), dtype=np.float64)
    p = mlp.unpack(flat, 40)
    assert p["E"].shape == (64, 40) and p["E"][0, 0] == 0
    assert p["b4"][0] == flat[-1]
    assert np.array_equal(mlp.pack(p, 40), flat)


def test_features():
    f = mlp.features([256, 8388608], [[32, 1, 1], [4, 8, 1]], np.arange(7) / 10)
    assert f.shape == (2, 16)
    assert f[0, 0] == 8 / 23 and f[1, 0] == 1.0
    assert f[0, 1] == 0.5 and f[1, 2] == 0.3 and f[1, 3] == 0.0
    assert np.all(f[:, 11:] == 0) and math.isclose(f[0, 10], 0.6)
