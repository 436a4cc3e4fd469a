"""Parity at the full batched size, in the launch configuration the throughput
benchmark times: 10,000 kernels x 8 metrics (80,000 fits with 50-2000 noisy
samples each, 82 M samples, coordinates as uint8 base-2 logarithms and FP32
values; DF32 moments, no refinement, FP32
coefficients), then the FP32 argmin over 64 sizes x 51 block shapes per kernel
(640,000 queries), each part captured in a CUDA graph and replayed.

The oracle cannot redo all of it in a test, so it checks what it can compute
one item at a time: a seeded sample of whole kernels' fits (all 8 metrics)
against the FP64 SVD fit, and a seeded sample of kernels' queries against the
oracle's rational program evaluated on the same coefficient table at the same
full launch size.  Properties that hold at any size are checked on every
output: fit statuses, the argmin's agreement with the evaluator's own table,
feasibility of every choice and the launch parameters.

Tolerances are those of the smaller parity tests (derived there): fitted
coefficients within 64 u eps_DF32 / gap plus the FP32 rounding of the output;
cycles within 1e-4 relative (FP32); argmin indices bit-exact where the
oracle's best-versus-runner-up margin exceeds 1e-6.
"""
import numpy as np
import pytest

import bench
import workloads as W
from oracle import rational
from tests import gpu_cases as G

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS_DF32 = 2.0 ** -44
SEED = 2024
CHECK_KERNELS = 32


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as klr
    wl = bench.WORKLOAD
    fb, q = bench.make_inputs(SEED)
    ctx = klr.Context(0)
    n_fits, n_q = fb.n_fits, len(q.sizes)
    ctx.reserve(n_fits, n_q)
    dev = torch.device("cuda", 0)
    off = torch.from_numpy(fb.offsets).to(dev)
    # the benchmark's sample format: uint8 base-2 logarithms (KLR_EXP8)
    x = torch.from_numpy(np.round(np.log2(fb.x)).astype(np.uint8)).to(dev)
    y = torch.from_numpy(fb.y).to(dev)
    qo, qn = torch.from_numpy(q.offsets).to(dev), torch.from_numpy(q.sizes).to(dev)
    regs = torch.from_numpy(fb.truth.regs).to(dev)
    smem = torch.from_numpy(fb.truth.smem).to(dev)
    cfg = torch.from_numpy(klr.enumerate_configs(2)).to(dev)
    hw = klr.make_hw(W.HARDWARE)
    m = klr._n_monomials(3, 2)
    coef = torch.empty((n_fits, 2 * m), device=dev, dtype=torch.float32)
    fst = torch.empty(n_fits, device=dev, dtype=torch.int32)
    fdg = torch.empty((n_fits, 4), device=dev, dtype=torch.float64)
    outs = [torch.empty(n_q, device=dev, dtype=t)
            for t in (torch.int32, torch.float32, torch.float32, torch.int32)]
    outs.append(torch.empty((n_q, 6), device=dev, dtype=torch.int32))
    truth_t = torch.from_numpy(fb.truth.coef.astype(np.float32)).to(dev)
    tout = [torch.empty_like(o) for o in outs]

    def prog_of(c):
        return klr.Context.program(c.view(wl["kernels"], 8, 2 * m), regs, smem, n_vars=3,
                                   degree=2, n_scale_log2=23, b_scale_log2=10,
                                   metric_lo=W.METRIC_LO, metric_scale=W.METRIC_SCALE)

    prog, prog_truth = prog_of(coef), prog_of(truth_t)

    def step():
        ctx.fit(off, x, y, n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10,
                precision=klr.FIT_DF32, refine_iters=0, coef_dtype=klr.F32,
                out=(coef, fst, fdg))
        ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32, out=tuple(outs))
        ctx.argmin(prog_truth, hw, cfg, qo, qn, out_dtype=klr.F32, out=tuple(tout))

    step()                                   # eager warm-up (workspace sized)
    torch.cuda.synchronize()
    for o in outs + tout + [coef, fst]:
        o.fill_(-7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    g.replay()
    torch.cuda.synchronize()
    table = ctx.eval(prog, hw, cfg, qo, qn, out_dtype=klr.F32)
    torch.cuda.synchronize()
    host = lambda ts: [t.cpu().numpy() for t in ts]
    return dict(klr=klr, fb=fb, q=q, coef=coef.cpu().numpy().astype(np.float64),
                fst=fst.cpu().numpy(), fit_out=host(outs), truth_out=host(tout),
                table=table.cpu().numpy())


def _kernels():
    return W.subsample_kernels(SEED + 17, bench.WORKLOAD["kernels"], CHECK_KERNELS)


def test_full_size_fits_match_oracle(run):
    fb, coef, fst = run["fb"], run["coef"], run["fst"]
    assert coef.shape == (80000, 20)
    # every fit of this workload is well posed: no flag but INEXACT may be set
    assert np.all((fst & ~8) == 0), np.unique(fst)
    assert np.all(np.isfinite(coef))
    fits = np.concatenate([8 * k + np.arange(8) for k in _kernels()])
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x.astype(np.float64),
                                     fb.y.astype(np.float64), 3, 2, 23, 10, fits=fits)
    for i, f in enumerate(fits):
        assert (int(fst[f]) & ~8) == int(ost[i])
        gap = max(od[i][1] ** 2 - od[i][0] ** 2, 1e-300)
        err = float(np.max(np.abs(coef[f] - oc[i])))
        assert err <= 64.0 * 20 * EPS_DF32 / gap + 2.0 ** -24, (f, err, gap)


def test_full_size_argmin_matches_oracle(run):
    fb, q = run["fb"], run["q"]
    best, cyc, margin, status, launch = run["truth_out"]
    assert best.shape == (640000,)
    ks = _kernels()
    rows = G.query_rows(q.offsets, ks)
    ref = G.oracle_choose(fb.truth.coef.astype(np.float32), fb.truth, q.offsets, q.sizes,
                          kernels=ks)
    ref["cycles"] = np.asarray(ref["cycles"]).reshape(len(rows), -1)
    ref["boundary"] = np.asarray(ref["boundary"]).reshape(len(rows), -1)
    ref["best"] = np.asarray(ref["best"])
    ref["best_cycles"] = np.asarray(ref["best_cycles"], dtype=np.float64)
    ref["margin"] = np.asarray(ref["margin"], dtype=np.float64)
    strict, loose = G.compare_argmin(best[rows], cyc[rows], ref, 1e-4, 1e-6, 1e-5)
    assert strict > 0.9 * len(rows)
    klr = run["klr"]
    assert np.array_equal((status[rows] & klr.Q_NONE_FEASIBLE) != 0, ref["best"] < 0)


def test_full_size_fitted_program_argmin_matches_oracle(run):
    """The whole chain at full size: the oracle's rational program evaluated
    on the library's own fitted FP32 coefficients (the table the argmin of
    the step used) for the checked kernels' 2,048 queries, against the
    library's choices of that step."""
    fb, q, coef = run["fb"], run["q"], run["coef"]
    best, cyc, margin, status, launch = run["fit_out"]
    ks = _kernels()
    rows = G.query_rows(q.offsets, ks)
    fitted = coef.astype(np.float32).reshape(-1, 8, 20)
    ref = G.oracle_choose(fitted, fb.truth, q.offsets, q.sizes, kernels=ks)
    ref["cycles"] = np.asarray(ref["cycles"]).reshape(len(rows), -1)
    ref["boundary"] = np.asarray(ref["boundary"]).reshape(len(rows), -1)
    ref["best"] = np.asarray(ref["best"])
    ref["best_cycles"] = np.asarray(ref["best_cycles"], dtype=np.float64)
    ref["margin"] = np.asarray(ref["margin"], dtype=np.float64)
    strict, loose = G.compare_argmin(best[rows], cyc[rows], ref, 1e-4, 1e-6, 1e-5)
    assert strict > 0.9 * len(rows)
    klr = run["klr"]
    assert np.array_equal((status[rows] & klr.Q_NONE_FEASIBLE) != 0, ref["best"] < 0)


def test_full_size_pipeline_properties(run):
    """On the whole output of the fitted program: every choice is feasible,
    its cycles are the evaluator's table minimum (within the FP32 near-tie
    window that is re-decided in FP64), and the launch parameters follow."""
    klr, q = run["klr"], run["q"]
    best, cyc, margin, status, launch = run["fit_out"]
    table = run["table"].astype(np.float64)
    assert table.shape == (640000, 51)
    fin = np.isfinite(table)
    none = ~fin.any(axis=1)
    assert np.array_equal(best < 0, none)
    assert np.array_equal((status & klr.Q_NONE_FEASIBLE) != 0, none)
    ok = ~none
    r = np.nonzero(ok)[0]
    tmin = np.min(np.where(fin, table, np.inf), axis=1)
    chosen = table[r, best[r]]
    assert np.all(np.isfinite(chosen))
    assert np.all(chosen <= tmin[r] * (1 + 1e-4))
    # the FP32 sweep reports the table's own value; a near-tie re-decided in
    # FP64 reports the FP64 value (within the FP32 evaluator's 1e-4)
    tie = (status[r] & klr.Q_TIE_RESOLVED) != 0
    assert np.array_equal(cyc[r][~tie], chosen[~tie].astype(np.float32))
    assert np.allclose(cyc[r][tie], chosen[tie], rtol=1e-4, atol=0)
    # the margin is the relative gap to the runner-up (>= 0)
    assert np.all(margin[r] >= 0)
    cfg = klr.enumerate_configs(2)
    b = cfg[best[r]]
    N = q.sizes[r]
    want = np.stack([-(-N // b[:, 0]), -(-N // b[:, 1]), np.ones_like(N), b[:, 0], b[:, 1],
                     b[:, 2]], axis=1)
    assert np.array_equal(launch[r].astype(np.int64), want)
    assert np.all(launch[none] == 0)
