"""GPU tests of the launch-shape autotuner (klr_autotune_fit,
klr_autotune_argmin, klr_tune_export / klr_tune_import).

Every candidate shape the tuner may pick is forced in turn (by importing it
for the problem class the tuner recorded) and checked against the FP64
oracle with the tolerances of the fit and argmin parity tests: a shape changes
how work is spread over threads, never what is computed, so the moments
kernel's block shapes and the evaluator's block sizes give bitwise-identical
outputs, and the solver's lanes per fit change only the order of its
double-word partial sums.
"""
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


def _fit(klr, ctx, fb, autotune=False):
    off = torch.tensor(fb.offsets).cuda()
    x = torch.tensor(np.ascontiguousarray(fb.x)).cuda()
    y = torch.tensor(fb.y).cuda()
    coef, st, _ = ctx.fit(off, x, y, n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10,
                          precision=klr.FIT_DF32, refine_iters=0, coef_dtype=klr.F64,
                          autotune=autotune)
    torch.cuda.synchronize()
    return coef.cpu().numpy(), st.cpu().numpy()


def test_autotune_fit_every_shape_matches_oracle(klr):
    ctx = klr.Context(0)
    fb = W.fit_batch(23, 24, (50, 2000), noise=0.01, dtype=np.float32)
    coef_t, st_t = _fit(klr, ctx, fb, autotune=True)
    choice, ms = ctx.last_tune
    assert (choice >> 4) in (0, 1, 2) and (choice & 15) in (0, 1, 2) and ms > 0
    table = ctx.tune_export()
    assert len(table) == 1 and table[0][1] == choice
    key = table[0][0]
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x.astype(np.float64), fb.y.astype(np.float64),
                                     3, 2, 23, 10)
    gap = np.maximum(od[:, 1] ** 2 - od[:, 0] ** 2, 1e-300)
    bound = 64.0 * 20 * 2.0 ** -44 / gap
    by_solver = {}
    for shape in [(w << 4) | s for w in range(3) for s in range(3)]:
        ctx.tune_import([(key, shape)])
        coef, st = _fit(klr, ctx, fb)
        assert np.array_equal(st & ~8, ost), shape
        err = np.max(np.abs(coef - oc), axis=1)
        assert np.all(err <= bound), (shape, err.max())
        # the moments block shape does not change a bit of the result
        prev = by_solver.setdefault(shape & 15, coef)
        assert np.array_equal(prev, coef), shape
        if shape == choice:
            assert np.array_equal(coef, coef_t) and np.array_equal(st, st_t)


def test_autotune_argmin_every_shape_is_bitwise_identical(klr):
    ctx = klr.Context(0)
    gt = G.make_program(6, 48)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(48, W.log_spaced_sizes(64))
    prog = G.gpu_program(klr, torch.tensor(coef).cuda(), gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    qo, qn = torch.tensor(q.offsets).cuda(), torch.tensor(q.sizes).cuda()
    host = lambda res: [r.cpu().numpy() for r in res]
    tuned = host(ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32, autotune=True))
    choice, ms = ctx.last_tune
    assert choice in (0, 1, 2, 3) and ms > 0
    (key, rec), = ctx.tune_export()
    assert rec == choice
    for shape in range(4):
        ctx.tune_import([(key, shape)])
        got = host(ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32))
        for a, b in zip(got, tuned):
            assert np.array_equal(a, b), shape
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    ref["cycles"] = ref["cycles"].reshape(len(q.sizes), -1)
    ref["boundary"] = ref["boundary"].reshape(len(q.sizes), -1)
    strict, _ = G.compare_argmin(tuned[0], tuned[1], ref, 1e-4, 1e-6, 1e-5)
    assert strict > 0


def test_autotune_refuses_graph_capture_and_bad_imports(klr):
    ctx = klr.Context(0)
    fb = W.fit_batch(24, 2, 100, dtype=np.float32)
    off = torch.tensor(fb.offsets).cuda()
    x = torch.tensor(np.ascontiguousarray(fb.x)).cuda()
    y = torch.tensor(fb.y).cuda()
    out = (torch.empty((16, 20), device="cuda", dtype=torch.float32),
           torch.empty(16, device="cuda", dtype=torch.int32),
           torch.empty((16, 4), device="cuda", dtype=torch.float64))
    kw = dict(n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10, precision=klr.FIT_DF32,
              coef_dtype=klr.F32, out=out)
    ctx.fit(off, x, y, **kw)                 # scratch sized before capturing
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(klr.KlrError) as e:
        with torch.cuda.graph(g):
            ctx.fit(off, x, y, autotune=True, **kw)
    assert e.value.status == klr.EINVAL
    torch.cuda.synchronize()
    assert ctx.tune_export() == []
    with pytest.raises(klr.KlrError):
        ctx.tune_import([(1, 256)])
    with pytest.raises(klr.KlrError):
        ctx.tune_import([(1, -1)])
    assert ctx.tune_export() == []
