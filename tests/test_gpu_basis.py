"""GPU parity of the per-variable degree-bound bases (Section V-E): fits and
programs in a box basis against the FP64 oracle, and the choice of basis by
held-out error against the oracle's rule on its own errors.

Tolerances are those of the fit and argmin parity tests (derived there);
held-out errors are compared within 1e-4 relative (they are RMS relative
prediction errors of nearly equal coefficient vectors), and the chosen basis
where no candidate lies within 1e-3 relative of the choice threshold."""
import numpy as np
import pytest

import workloads as W
from oracle import rational
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def klr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as k
    return k


@pytest.fixture(scope="module")
def ctx(klr):
    return klr.Context(0)


def _dev(fb):
    return (torch.tensor(fb.offsets).cuda(), torch.tensor(np.ascontiguousarray(fb.x)).cuda(),
            torch.tensor(fb.y).cuda())


@pytest.mark.parametrize("vd,mode", [((2, 1, 1), "df32"), ((3, 1, 1), "df32"), ((2, 1, 1), "fp64")])
def test_box_basis_fit_matches_oracle(klr, ctx, vd, mode):
    fb = W.fit_batch(61, 6, (100, 400), var_degree=vd, noise=0.01, dtype=np.float32)
    prec = klr.FIT_DF32 if mode == "df32" else klr.FIT_FP64
    coef, st, _ = ctx.fit(*_dev(fb), n_vars=3, degree=0, n_scale_log2=23, b_scale_log2=10,
                          precision=prec, coef_dtype=klr.F64, var_degree=vd)
    coef, st = coef.cpu().numpy(), st.cpu().numpy()
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x.astype(np.float64), fb.y.astype(np.float64),
                                     3, 0, 23, 10, var_degree=vd)
    u = oc.shape[1]
    assert coef.shape == oc.shape
    eps = 2.0 ** -44 if mode == "df32" else 2.0 ** -53
    for f in range(len(oc)):
        if ost[f] & rational.FIT_RANK_DEFICIENT:
            continue
        assert (int(st[f]) & ~8) == int(ost[f])
        gap = max(od[f][1] ** 2 - od[f][0] ** 2, 1e-300)
        assert np.max(np.abs(coef[f] - oc[f])) <= 64.0 * u * eps / gap, (f, gap)


def test_box_program_argmin_matches_oracle(klr, ctx):
    vd = (2, 1, 1)
    gt = W.ground_truth(62, 24, 3, 2, 8, 23, 10, var_degree=vd)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(24, W.log_spaced_sizes(64))
    prog = klr.Context.program(torch.tensor(coef).cuda(), torch.tensor(gt.regs).cuda(),
                               torch.tensor(gt.smem).cuda(), n_vars=3, degree=0, n_scale_log2=23,
                               b_scale_log2=10, metric_lo=W.METRIC_LO,
                               metric_scale=W.METRIC_SCALE, var_degree=vd)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    best, cyc, _, st, _ = ctx.argmin(prog, hw, cfg, torch.tensor(q.offsets).cuda(),
                                     torch.tensor(q.sizes).cuda(), out_dtype=klr.F32)
    torch.cuda.synchronize()
    from oracle import configs as ocfg, program as oprog
    ref = oprog.choose(dict(coef=coef.astype(np.float64), regs=gt.regs, smem=gt.smem, n_vars=3,
                            degree=0, n_scale_log2=23, b_scale_log2=10, metric_lo=W.METRIC_LO,
                            metric_scale=W.METRIC_SCALE, var_degree=vd),
                       W.HARDWARE, ocfg.enumerate_configs(2), q.offsets, q.sizes)
    ref["cycles"] = ref["cycles"].reshape(len(q.sizes), -1)
    ref["boundary"] = ref["boundary"].reshape(len(q.sizes), -1)
    strict, _ = G.compare_argmin(best.cpu().numpy(), cyc.cpu().numpy(), ref, 1e-4, 1e-6, 1e-5)
    assert strict > 0.9 * len(q.sizes)


def _split(fb, frac=0.7):
    """Per fit, the first frac of its samples for training, the rest held out."""
    off = fb.offsets
    tr_idx, ho_idx, tr_off, ho_off = [], [], [0], [0]
    for f in range(len(off) - 1):
        a, b = int(off[f]), int(off[f + 1])
        c = a + int(frac * (b - a))
        tr_idx.append(np.arange(a, c))
        ho_idx.append(np.arange(c, b))
        tr_off.append(tr_off[-1] + c - a)
        ho_off.append(ho_off[-1] + b - c)
    ti, hi = np.concatenate(tr_idx), np.concatenate(ho_idx)
    return ((np.array(tr_off, dtype=np.int64), fb.x[:, ti], fb.y[ti]),
            (np.array(ho_off, dtype=np.int64), fb.x[:, hi], fb.y[hi]))


def test_basis_selection_matches_oracle(klr, ctx):
    from paper_1911_02373_gb300 import basis
    fb = W.fit_batch(63, 8, (200, 600), var_degree=(2, 1, 1), noise=0.01, dtype=np.float32)
    (to, tx, ty), (ho, hx, hy) = _split(fb)
    cands = [(1, 1, 1), (2, 1, 1), (3, 1, 1), 2]
    d = lambda a: torch.tensor(np.ascontiguousarray(a)).cuda()
    choice, E, _ = basis.select_basis(ctx, (d(to), d(tx), d(ty)), (d(ho), d(hx), d(hy)), cands,
                                      n_vars=3, n_scale_log2=23, b_scale_log2=10)
    choice, E = choice.cpu().numpy(), E.cpu().numpy()
    Eo = np.zeros_like(E)
    gap = np.zeros_like(E)
    for j, c in enumerate(cands):
        kw = dict(var_degree=c) if not isinstance(c, int) else {}
        deg = c if isinstance(c, int) else 0
        oc, _, od = rational.fit_batch(to, tx.astype(np.float64), ty.astype(np.float64), 3, deg,
                                       23, 10, **kw)
        gap[:, j] = od[:, 1] ** 2 - od[:, 0] ** 2
        for f in range(len(oc)):
            a, b = int(ho[f]), int(ho[f + 1])
            Eo[f, j] = rational.relative_rms(oc[f], hx[:, a:b], hy[a:b], 3, deg, 23, 10,
                                             kw.get("var_degree"))
    # The fitted functions agree to the coefficient bound 64 u eps / gap of
    # the fit tests; held-out errors (RMS of ~1% noise) follow to about that
    # bound over the noise.  Typical agreement is far tighter.
    sizes = [8, 12, 16, 10]
    us = 2 * np.array(sizes)
    bound = 64 * us[None, :] * 2.0 ** -44 / np.maximum(gap, 1e-300)
    rel = np.abs(E - Eo) / Eo
    assert np.median(rel) < 1e-5
    firm = bound < 1e-4
    assert firm.mean() > 0.4
    assert np.all(rel[firm] < 1e-2)
    want = rational.choose_basis(Eo, sizes)
    clear = 0
    for f in range(len(want)):
        lim = Eo[f].min() * 1.05 + 1e-6
        # a clear decision: no error (GPU or oracle) within 2% of the threshold
        if np.all(np.abs(Eo[f] - lim) > 2e-2 * lim) and np.all(np.abs(E[f] - lim) > 2e-2 * lim):
            clear += 1
            assert choice[f] == want[f], (f, E[f], Eo[f])
    assert clear > 0.7 * len(want)
    # without noise the truth's box is the smallest candidate that predicts the
    # held-out samples (the smaller box and the total-degree basis of degree 2
    # lack terms of the truth, the larger box fits no better)
    fb0 = W.fit_batch(64, 8, (200, 600), var_degree=(2, 1, 1), dtype=np.float32)
    (to, tx, ty), (ho, hx, hy) = _split(fb0)
    choice0, E0, _ = basis.select_basis(ctx, (d(to), d(tx), d(ty)), (d(ho), d(hx), d(hy)), cands,
                                        n_vars=3, n_scale_log2=23, b_scale_log2=10)
    assert np.mean(choice0.cpu().numpy() == 1) > 0.9


def test_choose_basis_kernel_matches_the_oracle_rule(klr, ctx):
    """klr_choose_basis against oracle.rational.choose_basis on error tables
    with exact ties at the threshold (binary fractions: least * (1 + tol) +
    floor is exact), NaN and infinite errors, rows with nothing finite,
    candidates of equal size and errors within the floor of each other."""
    rng = np.random.default_rng(7)
    n_fits, n_cand = 4000, 6
    sizes = [10, 8, 16, 8, 20, 35]
    tol, floor = 0.25, 2.0 ** -20
    E = rng.uniform(0.5, 1.0, (n_fits, n_cand))
    E[rng.random(E.shape) < 0.3] *= 1.2
    lo = E.min(axis=1)
    lim = lo * (1 + tol) + floor
    hit = rng.random(E.shape) < 0.2                 # exactly at the threshold
    E[hit] = np.broadcast_to(lim[:, None], E.shape)[hit]
    E[:200] = np.round(E[:200] * 64) / 64           # many exact ties
    E[rng.random(E.shape) < 0.05] = np.nan
    E[rng.random(E.shape) < 0.05] = np.inf
    E[300:310] = np.nan                            # nothing finite
    E[310:320] = 1e-7 * rng.random((10, n_cand))   # all within the floor
    got = ctx.choose_basis(torch.tensor(E).cuda(), sizes, tol=tol, floor=floor).cpu().numpy()
    want = rational.choose_basis(E, sizes, tol=tol, floor=floor)
    assert np.array_equal(got, want)
    assert np.all(got[300:310] == -1)
    # bad arguments fail before anything runs
    with pytest.raises(klr.KlrError):
        ctx.choose_basis(torch.tensor(E).cuda(), sizes[:5] + [0], tol=tol, floor=floor)
    with pytest.raises(klr.KlrError):
        ctx.choose_basis(torch.tensor(E).cuda(), sizes, tol=-1.0, floor=floor)
