"""Shared set-up for the GPU parity tests: seeded programs and queries, the
library's results through the C ABI, and the oracle's on the same inputs."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import configs as ocfg
from oracle import program as oprog


def make_program(seed, n_kernels, n_vars=3, degree=2, n_hi_log2=23):
    gt = W.ground_truth(seed, n_kernels, n_vars, degree, 8, n_hi_log2, 10)
    return gt


def oracle_program(coef, gt):
    return dict(coef=np.asarray(coef, dtype=np.float64), regs=gt.regs, smem=gt.smem,
                n_vars=gt.n_vars, degree=gt.degree, n_scale_log2=gt.n_scale_log2,
                b_scale_log2=gt.b_scale_log2, metric_lo=W.METRIC_LO,
                metric_scale=W.METRIC_SCALE)


def gpu_program(klr, coef_t, gt, torch):
    return klr.Context.program(coef_t, torch.tensor(gt.regs).cuda(), torch.tensor(gt.smem).cuda(),
                               n_vars=gt.n_vars, degree=gt.degree,
                               n_scale_log2=gt.n_scale_log2, b_scale_log2=gt.b_scale_log2,
                               metric_lo=W.METRIC_LO, metric_scale=W.METRIC_SCALE)


def oracle_choose(coef, gt, q_offsets, q_sizes, kernels=None):
    cfgs = ocfg.enumerate_configs(gt.n_vars - 1)
    return oprog.choose(oracle_program(coef, gt), W.HARDWARE, cfgs, q_offsets, q_sizes, kernels)


def query_rows(q_offsets, kernels):
    return np.concatenate([np.arange(q_offsets[k], q_offsets[k + 1]) for k in kernels])


def compare_table(gpu_cycles, ref, rel_tol, boundary_tol):
    """Element-by-element cycles comparison.  Returns (n_compared, n_excluded,
    max relative error).  The usable pattern (finite vs +inf) must match
    exactly; values are compared where the oracle's branch decisions are
    farther than boundary_tol (relative) from their thresholds."""
    want = ref["cycles"]
    got = np.asarray(gpu_cycles, dtype=np.float64)
    assert got.shape == want.shape
    fin = np.isfinite(want)
    assert np.array_equal(np.isfinite(got), fin), "meaningful/usable pattern differs"
    robust = fin & (ref["boundary"] > boundary_tol)
    rel = np.abs(got[robust] - want[robust]) / np.abs(want[robust])
    mx = float(rel.max()) if rel.size else 0.0
    assert mx <= rel_tol, f"max relative cycles error {mx:.3e} > {rel_tol:.1e}"
    return int(robust.sum()), int((fin & ~robust).sum()), mx


def compare_argmin(best, best_cycles, ref, rel_tol, margin_tol=1e-6, boundary_tol=0.0):
    """Argmin indices bit-exact wherever the oracle's margin exceeds margin_tol
    (and its best configuration is not at a branch boundary); elsewhere the
    library's choice must be one of the oracle's near-optimal configurations."""
    best = np.asarray(best, dtype=np.int64)
    bc = np.asarray(best_cycles, dtype=np.float64)
    rb, rv, rm = ref["best"], ref["best_cycles"], ref["margin"]
    n = len(rb)
    rows = np.arange(n)
    bnd = np.where(rb >= 0, ref["boundary"][rows, np.maximum(rb, 0)], np.inf)
    strict = (rm > margin_tol) & (bnd > boundary_tol)
    none = rb < 0
    assert np.array_equal(best[none], rb[none]), "infeasible queries differ"
    bad = strict & (best != rb)
    assert not bad.any(), f"{bad.sum()} argmin mismatches, e.g. rows {np.nonzero(bad)[0][:5]}"
    loose = ~strict & ~none
    if loose.any():
        chosen = ref["cycles"][rows[loose], best[loose]]
        assert np.all(chosen <= rv[loose] * (1 + max(margin_tol, rel_tol) * 4)), "loose choice too far"
    ok = ~none
    rel = np.abs(bc[ok & strict] - rv[ok & strict]) / rv[ok & strict]
    if rel.size:
        assert rel.max() <= rel_tol, f"best cycles error {rel.max():.3e}"
    return int(strict.sum()), int(loose.sum())
