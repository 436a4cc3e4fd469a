"""Oracle: the learned proposer's network (test infrastructure only).

The paper has no learned component; this project adds a surrogate of the
rational program (a small MLP that predicts log cycles of a (kernel, N, block
shape) triple) to propose candidate shapes that the exact rational program then
re-ranks.  This module is the plain FP64 statement of that network, its loss,
its gradients and its optimiser, against which the GPU kernels are checked.

Network (all dense layers are y = x W^T + b, W stored out x in, row-major):
  emb = coef E^T                         coef: the kernel's 8 x 2m fitted
                                         coefficients (n_coef values), E: 64 x n_coef
  x0  = [features (16) | emb (64)]       features: log2 N / 23, log2 b0 / 10,
                                         log2 b1 / 10, log2 b2 / 10 (0 for 2D
                                         shapes), the 7-value hardware feature
                                         vector, 5 zeros
  a1 = gelu(x0 W1^T + b1)      W1: 256 x 80
  a2 = gelu(a1 W2^T + b2)      W2: 256 x 256
  a3 = gelu(a2 W3^T + b3)      W3: 256 x 256
  pred = a3 W4^T + b4          W4: n_out x 256
with gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) (the tanh form of
Hendrycks and Gimpel).

Two output forms share everything else:
* per row (n_out = 0, one output): a row is a (kernel, N, block shape) triple;
  loss = mean squared error of pred against the target.
* per query (n_out = |F| outputs): a row is a (kernel, N) query, the block
  shape does not enter the features (its three values are 0), output c
  predicts shape c; targets of shapes that are not meaningful are non-finite
  and masked: loss = sum over finite targets of (pred - target)^2 / their
  count.
Optimiser: AdamW (Loshchilov and Hutter) with bias correction and decoupled
weight decay applied to every parameter.

Parameter vector order: E, W1, b1, W2, b2, W3, b3, W4, b4.
"""
from __future__ import annotations

import math

import numpy as np

FEAT = 16
EMB = 64
IN = FEAT + EMB
H = 256
C_GELU = math.sqrt(2.0 / math.pi)


def shapes(n_coef: int, n_out: int = 0):
    k = max(1, n_out)
    return [("E", (EMB, n_coef)), ("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)),
            ("W3", (H, H)), ("b3", (H,)), ("W4", (k, H)), ("b4", (k,))]


def param_count(n_coef: int, n_out: int = 0) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n_coef, n_out))


def unpack(flat: np.ndarray, n_coef: int, n_out: int = 0) -> dict:
    out, o = {}, 0
    for name, s in shapes(n_coef, n_out):
        n = int(np.prod(s))
        out[name] = flat[o:o + n].reshape(s)
        o += n
    return out


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(C_GELU * (z + 0.044715 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(C_GELU * (z + 0.044715 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * C_GELU * (1.0 + 3 * 0.044715 * z * z)


def features(N, cfg_rows, hw_feat):
    """(n, 16) feature block for sizes N and block shapes cfg_rows (n, 3), or
    cfg_rows None for per-query rows (shape features 0)."""
    N = np.asarray(N, dtype=np.float64)
    f = np.zeros((len(N), FEAT))
    f[:, 0] = np.log2(N) / 23.0
    if cfg_rows is not None:
        f[:, 1:4] = np.log2(np.asarray(cfg_rows, dtype=np.float64)) / 10.0
    f[:, 4:11] = np.asarray(hw_feat, dtype=np.float64)[None, :]
    return f


def forward(p: dict, feat, coef_rows, per_query: bool = False):
    """Returns pred ((n,) per row, (n, n_out) per query) and the cache for
    backward."""
    emb = coef_rows @ p["E"].T
    x0 = np.hstack([feat, emb])
    z1 = x0 @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    z3 = a2 @ p["W3"].T + p["b3"]
    a3 = gelu(z3)
    pred = a3 @ p["W4"].T + p["b4"]
    if not per_query:
        pred = pred[:, 0]
    return pred, (coef_rows, x0, z1, a1, z2, a2, z3, a3)


def loss_and_grads(p: dict, feat, coef_rows, target):
    """Loss and the gradient of every parameter (dict of arrays).  target (n,)
    per row: mean squared error; target (n, n_out) per query: squared error
    summed over the finite targets, over their count."""
    target = np.asarray(target, dtype=np.float64)
    pred, (coef_rows, x0, z1, a1, z2, a2, z3, a3) = forward(p, feat, coef_rows,
                                                            per_query=target.ndim == 2)
    g = {}
    if target.ndim == 1:
        n = len(target)
        r = pred - target
        loss = float(np.mean(r * r))
        dpred = 2.0 * r / n
        g["W4"] = dpred[None, :] @ a3
        g["b4"] = np.array([dpred.sum()])
        da3 = np.outer(dpred, p["W4"][0])
    else:
        mask = np.isfinite(target)
        count = int(mask.sum())
        r = np.where(mask, pred - np.where(mask, target, 0.0), 0.0)
        loss = float(np.sum(r * r) / count)
        dpred = 2.0 * r / count
        g["W4"] = dpred.T @ a3
        g["b4"] = dpred.sum(0)
        da3 = dpred @ p["W4"]
    dz3 = da3 * gelu_grad(z3)
    g["W3"] = dz3.T @ a2
    g["b3"] = dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x0
    g["b1"] = dz1.sum(0)
    demb = (dz1 @ p["W1"])[:, FEAT:]
    g["E"] = demb.T @ coef_rows
    return loss, g


def pack(d: dict, n_coef: int, n_out: int = 0) -> np.ndarray:
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1)
                           for name, _ in shapes(n_coef, n_out)])


def adamw(param, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (step counts from 1); returns new (param, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    param = param - lr * (mh / (np.sqrt(vh) + eps) + wd * param)
    return param, m, v
