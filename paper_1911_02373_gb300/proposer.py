"""Learned proposer: training set, training loop and the propose-then-re-rank
argmin, all through the library's C ABI.

The surrogate network predicts per-query centred log2 cycles, either of a
(kernel, N, block shape) row (per-row form) or of every shape of a (kernel, N)
query at once (per-query form).  Its training targets come from the rational
program itself (klr_eval, then klr_mlp_query_targets).  At query time the
network proposes the k most promising meaningful shapes (klr_propose) and the
exact rational program re-ranks them (klr_argmin_candidates), so the plain
method remains the arbiter.  Random numbers (initial weights, training rows,
batch order) are inputs drawn by the caller.
"""
from __future__ import annotations

import math

import numpy as np

from . import F32, Context, Surrogate, argmin_candidates, mlp_param_count, query_targets

FEAT, EMB, IN, H = 16, 64, 80, 256


def init_params(n_coef: int, normals: np.ndarray, n_out: int = 0) -> np.ndarray:
    """Scale standard normals into initial parameters: weights ~ N(0, 1/fan_in)
    (E, W1..W3 with GELU gain 2, W4 with gain 1), biases zero."""
    n = mlp_param_count(n_coef, n_out)
    k = max(1, n_out)
    z = np.asarray(normals, dtype=np.float64)[:n].copy()
    shapes = [((EMB, n_coef), 1.0), ((H, IN), 2.0), ((H,), 0.0), ((H, H), 2.0), ((H,), 0.0),
              ((H, H), 2.0), ((H,), 0.0), ((k, H), 1.0), ((k,), 0.0)]
    o = 0
    for shape, gain in shapes:
        cnt = int(np.prod(shape))
        fan_in = shape[-1] if len(shape) == 2 else 1
        z[o:o + cnt] *= math.sqrt(gain / fan_in) if gain else 0.0
        o += cnt
    return z.astype(np.float32)


def query_table(ctx: Context, prog, hw, cfg, q_offsets, q_N):
    """(n_q, n_cfg) per-query centred log2 cycles from the FP32 rational
    program; NaN where a shape is not meaningful."""
    table = ctx.eval(prog, hw, cfg, q_offsets, q_N, out_dtype=F32)
    return query_targets(table)


def table_targets(ctx: Context, prog, hw, cfg, q_offsets, q_N, row_query, row_cfg):
    """Per-query centred log2 cycles of rows (query index, shape index);
    rows whose shape is not meaningful come back as NaN."""
    t = query_table(ctx, prog, hw, cfg, q_offsets, q_N)
    return t[row_query.long(), row_cfg.long()]


def train(sur: Surrogate, coef, cfg, kernel, N, cfg_idx, target, *, batch, epochs, lr,
          order, weight_decay=0.0, log_every=0):
    """Mini-batch AdamW over the rows for `epochs` passes.  order(epoch) gives
    the permutation of rows for that epoch (device int64).  Cosine learning-rate
    decay from lr.  A per-query network takes cfg_idx None and target
    (rows, n_out).  Returns the per-step losses (host floats)."""
    import torch
    n = kernel.numel()
    steps_per_epoch = max(1, (n + batch - 1) // batch)
    total = steps_per_epoch * epochs
    losses = []
    loss = torch.zeros(1, dtype=torch.float32, device=coef.device)
    step = 0
    for ep in range(epochs):
        perm = order(ep)
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            frac = step / max(1, total - 1)
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * frac))
            sur.train_step(coef, cfg, kernel[idx].contiguous(), N[idx].contiguous(),
                           None if cfg_idx is None else cfg_idx[idx].contiguous(),
                           target[idx].contiguous(), cur, weight_decay, True, loss)
            if log_every and step % log_every == 0:
                losses.append(float(loss.item()))
            step += 1
    losses.append(float(loss.item()))
    return losses


def propose_and_rerank(ctx: Context, sur: Surrogate, prog, hw, coef, regs, smem, cfg, q_offsets,
                       q_N, k):
    """The surrogate path: top-k proposal, then exact re-ranking.  Returns
    (best shape index, its FP32 cycles, status, candidates)."""
    cand = sur.propose(coef, regs, smem, hw, cfg, q_offsets, q_N, k)
    best, cyc, st = argmin_candidates(ctx, prog, hw, cfg, q_offsets, q_N, cand)
    return best, cyc, st, cand
