"""klr_argmin_noalloc: the argmin for callers that cannot allocate device memory.

Such callers -- a hook that picks launch parameters just before a kernel
launch, code running under CUDA graph capture, processes whose device memory
belongs to another allocator -- get an entry point whose scratch is a static
device array of the library.  This test calls it through the C ABI and checks it
against klr_argmin (context scratch) on the same inputs, for two calls in a row
with different inputs (the array keeps the previous call's contents, so the
second call also checks that the call clears what must start at zero).
Collected last on purpose; passes alone in a fresh process and after the other
tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _inputs(klr, seed, n_kernels, n_vars, sizes):
    gt = W.ground_truth(seed, n_kernels, n_vars, 2, 8, 23, 10)
    coef = torch.tensor(gt.coef.astype(np.float32)).cuda()
    prog = klr.Context.program(coef, torch.tensor(gt.regs).cuda(), torch.tensor(gt.smem).cuda(),
                               n_vars=n_vars, degree=2, n_scale_log2=23, b_scale_log2=10,
                               metric_lo=W.METRIC_LO, metric_scale=W.METRIC_SCALE)
    q = W.queries_per_kernel(n_kernels, sizes)
    cfg = torch.tensor(klr.enumerate_configs(n_vars - 1)).cuda()
    return prog, cfg, torch.tensor(q.offsets).cuda(), torch.tensor(q.sizes).cuda()


def test_noalloc_matches_context_argmin_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as klr
    ctx = klr.Context(0)
    hw = klr.make_hw(W.HARDWARE)
    cases = [(41, 600, 3, W.log_spaced_sizes(64)),      # 38,400 queries, 51 shapes
             (42, 40, 4, W.log_spaced_sizes(256))]      # 10,240 queries, 251 shapes
    for seed, nk, nv, sizes in cases:
        prog, cfg, qo, qn = _inputs(klr, seed, nk, nv, sizes)
        n = qn.numel()
        assert n <= klr.ARGMIN_NOALLOC_MAX_QUERIES
        # poison the outputs so stale values cannot pass
        out = (torch.full((n,), -7, dtype=torch.int32, device="cuda"),
               torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
               torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
               torch.full((n,), -1, dtype=torch.int32, device="cuda"),
               torch.full((n, 6), -1, dtype=torch.int32, device="cuda"))
        klr.argmin_noalloc(prog, hw, cfg, qo, qn, out)
        ref = ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32)
        torch.cuda.synchronize()
        best, cyc, margin, status, launch = [t.cpu().numpy() for t in out]
        rbest, rcyc, rmargin, rstatus, rlaunch = [t.cpu().numpy() for t in ref]
        assert np.array_equal(best, rbest)
        fin = np.isfinite(rcyc)
        assert np.array_equal(np.isfinite(cyc), fin)
        assert np.all(np.abs(cyc[fin] - rcyc[fin]) <= 1e-4 * np.abs(rcyc[fin]))
        assert np.array_equal(status, rstatus)
        assert np.array_equal(launch, rlaunch)
        ok = np.isfinite(rmargin)
        assert np.array_equal(np.isfinite(margin), ok)
        assert np.all(np.abs(margin[ok] - rmargin[ok]) <= 1e-4 * np.abs(rmargin[ok]) + 1e-7)
    # beyond the stated maximum: a clear error, nothing enqueued
    big = klr.ARGMIN_NOALLOC_MAX_QUERIES + 1
    prog, cfg, qo, qn = _inputs(klr, 43, 1, 3, np.full(big, 4096, dtype=np.int64))
    out = tuple(torch.empty(s, dtype=d, device="cuda") for s, d in
                [((big,), torch.int32), ((big,), torch.float32), ((big,), torch.float32),
                 ((big,), torch.int32), ((big, 6), torch.int32)])
    with pytest.raises(klr.KlrError) as e:
        klr.argmin_noalloc(prog, hw, cfg, qo, qn, out)
    assert e.value.status == klr.EINVAL and "maximum" in str(e.value)
    ctx.close()


def test_noalloc_more_near_ties_than_its_tie_records():
    """More FP32 near-ties than the static array holds tie records for: the
    queries past its KLR_ARGMIN_NOALLOC_TIE_RECORDS are re-decided in FP64
    in place by the sweep instead of by the tie passes.  Both routes must
    give what klr_argmin (whose context scratch lists every one of them)
    gives, bit for bit.  The program's metrics do not depend on the block
    shape, so every shape of a thread count has the same cycles and every
    query is a near-tie."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    import os
    import paper_1911_02373_gb300 as klr
    with open(os.path.join(os.path.dirname(__file__), "golden", "chain_cases.json")) as f:
        g = json.load(f)
    k = g["kernels"]["B"]           # constant metrics
    coef = torch.tensor(np.array(k["coef"], dtype=np.float32)[None]).cuda()
    prog = klr.Context.program(coef, torch.tensor([k["regs"]], dtype=torch.int32).cuda(),
                               torch.tensor([k["smem"]], dtype=torch.int32).cuda(), n_vars=3,
                               degree=2, n_scale_log2=23, b_scale_log2=10,
                               metric_lo=g["metric_lo"], metric_scale=g["metric_scale"])
    n = klr.ARGMIN_NOALLOC_TIE_RECORDS + 7616
    u = W.uniform(W.stream_key(44, 1), np.arange(n, dtype=np.uint64))
    sizes = np.floor(np.exp2(10 + 12 * u)).astype(np.int64)
    qo = torch.tensor([0, n], dtype=torch.int64).cuda()
    qn = torch.tensor(sizes).cuda()
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    hw = klr.make_hw(g["hw"])
    ctx = klr.Context(0)
    out = (torch.full((n,), -7, dtype=torch.int32, device="cuda"),
           torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
           torch.full((n,), -1.0, dtype=torch.float32, device="cuda"),
           torch.full((n,), -1, dtype=torch.int32, device="cuda"),
           torch.full((n, 6), -1, dtype=torch.int32, device="cuda"))
    klr.argmin_noalloc(prog, hw, cfg, qo, qn, out)
    ref = ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=klr.F32)
    torch.cuda.synchronize()
    got = [t.cpu().numpy() for t in out]
    want = [t.cpu().numpy() for t in ref]
    tied = (want[3] & klr.Q_TIE_RESOLVED) != 0
    assert tied.sum() > klr.ARGMIN_NOALLOC_TIE_RECORDS, tied.sum()
    assert np.array_equal(got[3], want[3])
    assert np.array_equal(got[0], want[0]) and np.all(got[0] >= 0)
    assert np.array_equal(got[1].view(np.int32), want[1].view(np.int32))
    assert np.array_equal(got[2].view(np.int32), want[2].view(np.int32))
    assert np.array_equal(got[4], want[4])
    ctx.close()
