"""The hand-worked whole-chain cases (tests/golden/chain_cases.json) through
the library: klr_argmin (FP32 with FP64 near-ties, and FP64) and klr_eval,
compared with the values worked by hand from Section IV, steps 4-5 -- not
with the oracle -- so a mistake shared by the oracle and the kernels would
still show here."""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chain_cases.json")


def _setup(torch, klr, g, name, sizes):
    k = g["kernels"][name]
    coef = torch.tensor(np.array(k["coef"], dtype=np.float64)[None]).cuda()
    regs = torch.tensor([k["regs"]], dtype=torch.int32).cuda()
    smem = torch.tensor([k["smem"]], dtype=torch.int32).cuda()
    qo = torch.tensor([0, len(sizes)], dtype=torch.int64).cuda()
    qn = torch.tensor(sizes, dtype=torch.int64).cuda()
    return coef, regs, smem, qo, qn


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_chain_golden_argmin(dtype):
    torch = pytest.importorskip("torch")
    import paper_1911_02373_gb300 as klr
    with open(GOLDEN) as f:
        g = json.load(f)
    ctx = klr.Context(0)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    hw = klr.make_hw(g["hw"])
    F = [tuple(int(v) for v in r[:2]) for r in klr.enumerate_configs(2)]
    rel = 1e-6 if dtype == "f32" else 1e-12
    for name in g["kernels"]:
        cases = [c for c in g["queries"] if c["kernel"] == name]
        if not cases:
            continue
        sizes = [c["N"] for c in cases]
        coef, regs, smem, qo, qn = _setup(torch, klr, g, name, sizes)
        if dtype == "f32":
            coef = coef.float()
        prog = klr.Context.program(coef, regs, smem, n_vars=g["n_vars"], degree=g["degree"],
                                   n_scale_log2=g["n_scale_log2"], b_scale_log2=g["b_scale_log2"],
                                   metric_lo=g["metric_lo"], metric_scale=g["metric_scale"])
        best, cyc, mrg, st, lp = ctx.argmin(prog, hw, cfg, qo, qn,
                                            out_dtype=klr.F32 if dtype == "f32" else klr.F64)
        torch.cuda.synchronize()
        best, cyc, mrg = best.cpu().numpy(), cyc.cpu().numpy(), mrg.cpu().numpy()
        st, lp = st.cpu().numpy(), lp.cpu().numpy()
        for i, c in enumerate(cases):
            tag = f'{name} N={c["N"]} {dtype}'
            assert best[i] == c["best"], tag
            assert (st[i] & 3) == c["status"], tag
            if c["best"] < 0:
                continue
            assert F[c["best"]] == tuple(c["best_config"]), tag
            assert cyc[i] == pytest.approx(c["best_cycles"], rel=rel), tag
            assert mrg[i] == pytest.approx(c["margin"], rel=1e-4, abs=1e-7), tag
            b0, b1 = c["best_config"]
            N = c["N"]
            assert tuple(lp[i]) == (-(-N // b0), -(-N // b1), 1, b0, b1, 1), tag
    ctx.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_chain_golden_cells(dtype):
    torch = pytest.importorskip("torch")
    import paper_1911_02373_gb300 as klr
    with open(GOLDEN) as f:
        g = json.load(f)
    ctx = klr.Context(0)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    hw = klr.make_hw(g["hw"])
    F = [tuple(int(v) for v in r[:2]) for r in klr.enumerate_configs(2)]
    rel = 1e-6 if dtype == "f32" else 1e-12
    for c in g["cells"]:
        coef, regs, smem, qo, qn = _setup(torch, klr, g, c["kernel"], [c["N"]])
        if dtype == "f32":
            coef = coef.float()
        prog = klr.Context.program(coef, regs, smem, n_vars=g["n_vars"], degree=g["degree"],
                                   n_scale_log2=g["n_scale_log2"], b_scale_log2=g["b_scale_log2"],
                                   metric_lo=g["metric_lo"], metric_scale=g["metric_scale"])
        table = ctx.eval(prog, hw, cfg, qo, qn,
                         out_dtype=klr.F32 if dtype == "f32" else klr.F64).cpu().numpy()
        got = float(table[0, F.index(tuple(c["config"]))])
        tag = f'{c["kernel"]} N={c["N"]} b={c["config"]} {dtype}'
        if c["cycles"] is None:
            assert not math.isfinite(got), tag
        else:
            assert got == pytest.approx(c["cycles"], rel=rel), tag
    ctx.close()
