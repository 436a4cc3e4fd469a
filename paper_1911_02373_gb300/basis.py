"""Choosing the monomial basis of each fit by held-out error.

Section V-E bounds the degree of each variable separately and leaves the
bounds to be chosen; here every candidate basis (per-variable bounds, or a
total degree) is fitted on the training samples (klr_fit) and scored on
held-out samples of the same fits (klr_fit_heldout).  Per fit the smallest
basis whose held-out RMS relative error is within (1 + tol) of the least,
plus an absolute floor (errors below it count as equal; the default 1e-6 is
above the relative rounding of FP32 samples), is chosen (ties: the earlier
candidate).
"""
from __future__ import annotations

from . import F64, FIT_DF32, Context, _n_monomials


def select_basis(ctx: Context, train, heldout, candidates, *, n_vars, n_scale_log2,
                 b_scale_log2, precision=FIT_DF32, refine_iters=0, tol=0.05, floor=1e-6):
    """train, heldout: (offsets, x, y) CSR sample sets of the same fits.
    candidates: per-variable bound tuples, or ints (total degree).
    Returns (choice (n_fits,) int32 device tensor from klr_choose_basis, -1
    where no candidate has a finite error; errors (n_fits, n_cand) float64;
    coefficients per candidate)."""
    import torch
    errs, coefs, sizes = [], [], []
    for cand in candidates:
        kw = dict(degree=cand, var_degree=None) if isinstance(cand, int) else \
            dict(degree=0, var_degree=tuple(cand))
        coef, _, _ = ctx.fit(*train, n_vars=n_vars, n_scale_log2=n_scale_log2,
                             b_scale_log2=b_scale_log2, precision=precision,
                             refine_iters=refine_iters, coef_dtype=F64, **kw)
        errs.append(ctx.fit_heldout(*heldout, coef, n_vars=n_vars, n_scale_log2=n_scale_log2,
                                    b_scale_log2=b_scale_log2, **kw))
        coefs.append(coef)
        sizes.append(_n_monomials(n_vars, kw["degree"], kw["var_degree"]))
    E = torch.stack(errs, dim=1).contiguous()
    choice = ctx.choose_basis(E, sizes, tol=tol, floor=floor)
    return choice, E, coefs
