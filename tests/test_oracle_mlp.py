"""Pins of the surrogate network's oracle: analytic gradients against central
finite differences (FP64), GELU against its defining formula's limits and
derivative and against the exact form z Phi(z) it approximates, AdamW's first
step against its closed form.  A mutation test reruns these pins on private
copies of ``oracle.mlp`` with one plausible mistake planted at a time."""
import math
import os
import sys
import types

import numpy as np
import pytest

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


def test_gelu_is_near_the_exact_form():
    # the tanh form approximates z Phi(z) (Phi the standard normal CDF, here
    # from math.erf): within 4.8e-4 everywhere on [-8, 8]; a wrong constant
    # (sqrt(1/pi) or 2/pi for sqrt(2/pi), no cubic term) misses by 0.03-0.1
    z = np.linspace(-8.0, 8.0, 3201)
    exact = np.array([v * 0.5 * (1.0 + math.erf(v / math.sqrt(2.0))) for v in z])
    assert np.max(np.abs(mlp.gelu(z) - exact)) <= 5e-4


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


def _tiny_head(seed=2, n=6, n_coef=24, n_out=5):
    rng = np.random.default_rng(seed)
    flat = rng.standard_normal(mlp.param_count(n_coef, n_out)) * 0.2
    feat = mlp.features(2.0 ** rng.uniform(8, 23, n), None, rng.standard_normal(7) * 0.3)
    coef = rng.standard_normal((n, n_coef)) * 0.3
    target = rng.standard_normal((n, n_out))
    target[rng.random((n, n_out)) < 0.3] = np.inf          # shapes that are not meaningful
    return flat, feat, coef, target


def test_per_query_head_gradients_match_finite_differences():
    n_coef, n_out = 24, 5
    flat, feat, coef, target = _tiny_head(n_coef=n_coef, n_out=n_out)
    assert np.all(feat[:, 1:4] == 0.0)
    p = mlp.unpack(flat, n_coef, n_out)
    loss, g = mlp.loss_and_grads(p, feat, coef, target)
    gflat = mlp.pack(g, n_coef, n_out)
    assert gflat.shape == flat.shape
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(len(flat), 50, replace=False),
                          np.arange(len(flat) - 6 * 256 - 5, len(flat))[::97]])
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unpack(fp, n_coef, n_out), feat, coef, target)
        lm, _ = mlp.loss_and_grads(mlp.unpack(fm, n_coef, n_out), feat, coef, target)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_per_query_head_masked_loss():
    n_coef, n_out = 24, 5
    flat, feat, coef, target = _tiny_head(n_coef=n_coef, n_out=n_out)
    p = mlp.unpack(flat, n_coef, n_out)
    pred, _ = mlp.forward(p, feat, coef, per_query=True)
    mask = np.isfinite(target)
    loss, g = mlp.loss_and_grads(p, feat, coef, target)
    # the loss is the mean squared error over the finite targets only
    assert np.isclose(loss, np.mean((pred[mask] - target[mask]) ** 2), rtol=1e-14)
    # a masked output receives no gradient through its row of W4 and b4
    masked_cols = np.nonzero(~mask.any(axis=0))[0]
    for c in masked_cols:
        assert np.all(g["W4"][c] == 0.0) and g["b4"][c] == 0.0
    # changing a masked target changes nothing
    t2 = target.copy()
    t2[~mask] = -np.inf
    loss2, g2 = mlp.loss_and_grads(p, feat, coef, t2)
    assert loss2 == loss and np.array_equal(mlp.pack(g2, n_coef, n_out), mlp.pack(g, n_coef, n_out))
    # with every target finite, one output column and zero shape features the
    # per-query form is the per-row form on the same rows
    flat1 = flat[:mlp.param_count(n_coef, 1)]
    p1 = mlp.unpack(flat1, n_coef, 1)
    t1 = np.random.default_rng(4).standard_normal((len(feat), 1))
    lq, gq = mlp.loss_and_grads(p1, feat, coef, t1)
    lr_, gr = mlp.loss_and_grads(p1, feat, coef, t1[:, 0])
    assert np.isclose(lq, lr_, rtol=1e-14)
    assert np.allclose(mlp.pack(gq, n_coef, 1), mlp.pack(gr, n_coef, 0), rtol=1e-12, atol=1e-15)


# --- planted mistakes ------------------------------------------------------------

# (original text in oracle/mlp.py, planted mistake)
MLP_MUTATIONS = [
    ("C_GELU = math.sqrt(2.0 / math.pi)", "C_GELU = math.sqrt(1.0 / math.pi)"),
    ("    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))",
     "    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.04715 * z ** 3)))"),
    ("    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * z * z)",
     "    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU"),
    ("    a2 = gelu(z2)", "    a2 = z2"),
    ("    dz2 = (dz3 @ p[\"W3\"]) * gelu_grad(z2)", "    dz2 = (dz3 @ p[\"W3\"].T) * gelu_grad(z2)"),
    ("    demb = (dz1 @ p[\"W1\"])[:, FEAT:]", "    demb = (dz1 @ p[\"W1\"])[:, :EMB]"),
    ("        dpred = 2.0 * r / n", "        dpred = r / n"),
    ("        loss = float(np.sum(r * r) / count)", "        loss = float(np.sum(r * r) / r.size)"),
    ("        r = np.where(mask, pred - np.where(mask, target, 0.0), 0.0)",
     "        r = np.where(mask, pred - np.where(mask, target, 0.0), pred)"),
    ("    mh = m / (1 - beta1 ** step)", "    mh = m"),
    ("    param = param - lr * (mh / (np.sqrt(vh) + eps) + wd * param)",
     "    param = param - lr * (mh / (np.sqrt(vh) + eps) - wd * param)"),
    ("    f[:, 0] = np.log2(N) / 23.0", "    f[:, 0] = np.log2(N) / 24.0"),
]

PINS = [test_gradients_match_finite_differences, test_gelu_limits_and_derivative,
        test_gelu_is_near_the_exact_form, test_adamw_first_step_closed_form,
        test_parameter_layout, test_features,
        test_per_query_head_gradients_match_finite_differences,
        test_per_query_head_masked_loss]


def _pins_failing_on(module, monkeypatch):
    """Names of the pins above that fail with ``module`` in place of oracle.mlp."""
    monkeypatch.setattr(sys.modules[__name__], "mlp", module)
    failed = []
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:  # an assertion or a crash: the pin noticed
            failed.append(pin.__name__)
    return failed


def test_mlp_pins_pass_on_the_oracle(monkeypatch):
    assert _pins_failing_on(mlp, monkeypatch) == []


@pytest.mark.parametrize("orig,planted", MLP_MUTATIONS)
def test_mlp_pins_catch_planted_mistakes(orig, planted, monkeypatch):
    path = mlp.__file__
    src = open(path).read()
    assert src.count(orig) == 1, f"{os.path.basename(path)} no longer holds {orig!r} once"
    mod = types.ModuleType("oracle._planted_mlp")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, planted), path + " (planted)", "exec"), mod.__dict__)
    assert _pins_failing_on(mod, monkeypatch), f"no pin notices {planted!r}"
