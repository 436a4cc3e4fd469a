"""Oracle: the rational program and the choice of launch parameters
(test infrastructure only).

Section IV, steps 4 and 5: at run time, for the given data parameters and for
every practically meaningful configuration in F, evaluate the rational program
(fitted low-level metrics -> occupancy -> MWP-CWP cycles) and select the
configuration that minimises the estimate.  The paper's IO function returns the
six launch integers (gx, gy, gz, bx, by, bz) (Section V-C), with grid sizes
ceil(N / b) (Section V-A).

Readings of this project:
* metric i of a kernel is L_i = lo_i + s_i |p_i(x) / q_i(x)| (a rational
  program per Definition 1's extensions; |.| is a comparison);  q_i(x) = 0 or a
  non-finite value makes that configuration unusable for the query (flag bit 1);
* a configuration is meaningful (footnote to step 4) when B_active > 0,
  T <= T_max and every block dimension b_i <= N;
* ties go to the lowest configuration index; no configuration -> index -1;
* margin = (runner-up - best) / best over meaningful configurations (+inf with a
  single one, 0 with none);
* the secondary-metric refinement of step 5 is not applied (the paper leaves it
  unspecified).
"""
from __future__ import annotations

import math

import numpy as np

from . import mwpcwp, occupancy, rational

Q_OK = 0
Q_BAD_METRIC = 1     # q = 0 or non-finite metric at some configuration
Q_NONE_FEASIBLE = 2  # no meaningful configuration


def metrics(coef8: np.ndarray, xs: np.ndarray, exps: list, lo, scale):
    """L (8, ...) and validity (...) at scaled points xs (..., n_vars)."""
    m = len(exps)
    phi = rational.monomials(xs, exps)                   # (..., m)
    p = np.einsum("...t,it->i...", phi, coef8[:, :m])    # (8, ...)
    q = np.einsum("...t,it->i...", phi, coef8[:, m:])
    with np.errstate(divide="ignore", invalid="ignore"):
        g = p / q
    valid = np.all((q != 0) & np.isfinite(g), axis=0)
    lo = np.asarray(lo, dtype=np.float64).reshape((8,) + (1,) * (g.ndim - 1))
    sc = np.asarray(scale, dtype=np.float64).reshape((8,) + (1,) * (g.ndim - 1))
    return lo + sc * np.abs(g), valid


def kernel_occupancy(regs: int, smem: int, configs, hw):
    """(B_active, W_active) per configuration for one kernel (integers)."""
    # Python integers throughout: the products in Fig. 1's tests exceed 32 bits
    T = [int(math.prod(int(v) for v in c)) for c in configs]
    B = np.array([occupancy.active_blocks(t, int(regs), int(smem), hw) for t in T],
                 dtype=np.int64)
    W = np.array([occupancy.active_warps(int(b), t, hw) for b, t in zip(B, T)], dtype=np.int64)
    return B, W


def evaluate_kernel(coef8, regs, smem, sizes, configs, hw, metric_lo, metric_scale,
                    n_vars, degree, n_scale_log2, b_scale_log2, var_degree=None):
    """Cycles of every (query size, configuration) of one kernel.

    Returns dict of arrays shaped (n_sizes, n_cfg): cycles (inf where not
    meaningful or invalid), meaningful, valid, branch, boundary (margin of the
    branch decisions)."""
    exps = rational.monomial_exponents(n_vars, degree, var_degree)
    cfg = np.array(configs, dtype=np.int64)                  # (C, dims)
    N = np.asarray(sizes, dtype=np.int64)                    # (Q,)
    T = np.prod(cfg, axis=1)                                 # (C,)
    B, W = kernel_occupancy(regs, smem, configs, hw)
    meaningful = ((B > 0)[None, :] & (T <= hw["max_threads_per_block"])[None, :]
                  & np.all(cfg[None, :, :] <= N[:, None, None], axis=2))
    raw = np.empty(N.shape + (len(configs), n_vars))
    raw[..., 0] = N[:, None].astype(np.float64)
    raw[..., 1:] = cfg[None, :, :].astype(np.float64)
    xs = rational.scale_variables(raw, n_scale_log2, b_scale_log2)
    L, valid = metrics(np.asarray(coef8, dtype=np.float64), xs, exps,
                       metric_lo, metric_scale)
    n_blocks = -(-N[:, None] // T[None, :])                  # ceil(N / T), exact
    active_sms = np.minimum(hw["n_sm"], n_blocks)
    per_wave = np.maximum(B[None, :] * active_sms, 1)
    rep = -(-n_blocks // per_wave)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        e, branch, boundary = mwpcwp.cycles(
            [L[i] for i in range(8)], hw, np.broadcast_to(W[None, :], N.shape + W.shape),
            np.broadcast_to(B[None, :], N.shape + B.shape), active_sms, rep)
    usable = meaningful & valid
    return dict(cycles=np.where(usable, e, np.inf), meaningful=meaningful, valid=valid,
                branch=branch, boundary=boundary, B_active=B, W_active=W,
                n_blocks=n_blocks, rep=rep)


def argmin(cycles: np.ndarray):
    """Best index (lowest on ties), best value and relative margin, per row."""
    cycles = np.atleast_2d(cycles)
    best = np.full(cycles.shape[0], -1, dtype=np.int64)
    val = np.full(cycles.shape[0], np.inf)
    margin = np.zeros(cycles.shape[0])
    for r in range(cycles.shape[0]):
        row = cycles[r]
        fin = np.isfinite(row)
        if not fin.any():
            continue
        i = int(np.argmin(np.where(fin, row, np.inf)))  # first minimum
        best[r], val[r] = i, row[i]
        rest = np.delete(row, i)
        rest = rest[np.isfinite(rest)]
        margin[r] = (rest.min() - row[i]) / row[i] if rest.size else np.inf
    return best, val, margin


def refine(cycles: np.ndarray, warps: np.ndarray, eps: float):
    """Section IV, step 5's refinement among near-optimal configurations.

    The paper allows a secondary performance metric to choose among the
    configurations that optimise the estimate up to some margin, and names
    hardware occupancy among the performance metrics; it fixes neither the
    margin nor the metric.  Reading: among the configurations with cycles
    <= (1 + eps) x the least cycles, take the one with the most active warps
    per SM; ties by fewer cycles, then by the lower index.

    cycles: (Q, C) with inf where not meaningful; warps: (Q, C) or (C,)
    W_active.  Returns best index per row (-1 when nothing is finite)."""
    cycles = np.atleast_2d(cycles)
    warps = np.broadcast_to(warps, cycles.shape)
    best = np.full(cycles.shape[0], -1, dtype=np.int64)
    for r in range(cycles.shape[0]):
        row = cycles[r]
        fin = np.isfinite(row)
        if not fin.any():
            continue
        lo = row[fin].min()
        near = [c for c in range(len(row)) if fin[c] and row[c] <= lo * (1.0 + eps)]
        best[r] = min(near, key=lambda c: (-int(warps[r, c]), row[c], c))
    return best


def launch_params(best_cfg, N: int):
    """(gx, gy, gz, bx, by, bz): block shape and grid = ceil(N / b_i) per used
    dimension (Section V-A's grid file for square data), 1 elsewhere."""
    b = list(best_cfg) + [1] * (3 - len(best_cfg))
    g = [-(-N // bi) for bi in best_cfg] + [1] * (3 - len(best_cfg))
    return tuple(g) + tuple(b)


def choose(program: dict, hw: dict, configs, q_offsets, q_sizes, kernels=None):
    """Steps 4-5 for every query of the CSR query list (or kernel subset).

    program: dict(coef (K, 8, 2m), regs (K,), smem (K,), n_vars, degree,
    n_scale_log2, b_scale_log2, metric_lo, metric_scale).
    Returns dict with per-query best, best_cycles, margin, status and the
    per-query (n_cfg,) cycles table and boundary margins."""
    kernels = range(len(q_offsets) - 1) if kernels is None else kernels
    out = dict(best=[], best_cycles=[], margin=[], status=[], cycles=[], boundary=[],
               branch=[], kernel=[], size=[])
    for k in kernels:
        a, b = int(q_offsets[k]), int(q_offsets[k + 1])
        if a == b:
            continue
        ev = evaluate_kernel(program["coef"][k], program["regs"][k], program["smem"][k],
                             q_sizes[a:b], configs, hw, program["metric_lo"],
                             program["metric_scale"], program["n_vars"], program["degree"],
                             program["n_scale_log2"], program["b_scale_log2"],
                             program.get("var_degree"))
        best, val, margin = argmin(ev["cycles"])
        st = np.where(np.any(ev["meaningful"] & ~ev["valid"], axis=1), Q_BAD_METRIC, Q_OK)
        st = st | np.where(best < 0, Q_NONE_FEASIBLE, 0)
        out["best"].append(best)
        out["best_cycles"].append(val)
        out["margin"].append(margin)
        out["status"].append(st)
        out["cycles"].append(ev["cycles"])
        out["boundary"].append(np.where(ev["meaningful"], ev["boundary"], np.inf))
        out["branch"].append(ev["branch"])
        out["kernel"].append(np.full(b - a, k))
        out["size"].append(np.asarray(q_sizes[a:b]))
    return {key: (np.concatenate(v) if v else np.zeros(0)) for key, v in out.items()}
