"""GPU parity of the evaluator (E1-E5) against the FP64 oracle, through the C ABI.

Tolerances (stated by the design): cycles within 1e-4 relative for the FP32
evaluator and 1e-10 for the FP64 one, compared where the oracle's branch
decisions are clear of their thresholds (a piecewise boundary can flip between
precisions; those points are counted, not compared); the usable pattern
(occupancy > 0, T <= T_max, b_i <= N, valid metrics) bit-exact; argmin indices
bit-exact wherever the oracle's best-versus-runner-up margin exceeds 1e-6.
"""
import numpy as np
import pytest

import workloads as W
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


def _run(klr, ctx, gt, coef, q_offsets, q_sizes, dtype, table):
    ct = torch.tensor(coef).cuda()
    prog = G.gpu_program(klr, ct, gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(gt.n_vars - 1)).cuda()
    qo = torch.tensor(q_offsets).cuda()
    qn = torch.tensor(q_sizes).cuda()
    if table:
        out = ctx.eval(prog, hw, cfg, qo, qn, out_dtype=dtype)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    res = ctx.argmin(prog, hw, cfg, qo, qn, out_dtype=dtype)
    torch.cuda.synchronize()
    return [None if r is None else r.cpu().numpy() for r in res]


CASES = [
    # (name, seed, kernels, n_vars, sizes)
    ("single_2d", 5, 1, 3, W.query_sizes("pow2", 16)),
    ("batched_2d", 6, 48, 3, W.log_spaced_sizes(64)),
    ("sweep_3d", 7, 6, 4, W.log_spaced_sizes(256)),
    ("ragged_small_N", 8, 9, 3, np.array([1, 2, 17, 31, 32, 33, 100, 1000, 65537, 1 << 23])),
]


@pytest.mark.parametrize("name,seed,nk,nv,sizes", CASES)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_table_matches_oracle(klr, ctx, name, seed, nk, nv, sizes, dtype):
    gt = G.make_program(seed, nk, n_vars=nv)
    coef = gt.coef.astype(np.float32 if dtype == "f32" else np.float64)
    q = W.queries_per_kernel(nk, sizes)
    got = _run(klr, ctx, gt, coef, q.offsets, q.sizes, klr.F32 if dtype == "f32" else klr.F64, True)
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    want = np.stack(ref["cycles"]) if isinstance(ref["cycles"], list) else ref["cycles"]
    ref = dict(ref, cycles=want.reshape(len(q.sizes), -1),
               boundary=ref["boundary"].reshape(len(q.sizes), -1))
    tol, btol = (1e-4, 1e-5) if dtype == "f32" else (1e-10, 1e-12)
    n, excl, mx = G.compare_table(got, ref, tol, btol)
    assert n > 0 and excl <= 0.01 * n + 5


@pytest.mark.parametrize("name,seed,nk,nv,sizes", CASES)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_argmin_matches_oracle(klr, ctx, name, seed, nk, nv, sizes, dtype):
    gt = G.make_program(seed, nk, n_vars=nv)
    coef = gt.coef.astype(np.float32 if dtype == "f32" else np.float64)
    q = W.queries_per_kernel(nk, sizes)
    best, cyc, margin, status, launch = _run(klr, ctx, gt, coef, q.offsets, q.sizes,
                                             klr.F32 if dtype == "f32" else klr.F64, False)
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    ref["cycles"] = ref["cycles"].reshape(len(q.sizes), -1)
    ref["boundary"] = ref["boundary"].reshape(len(q.sizes), -1)
    tol, btol = (1e-4, 1e-5) if dtype == "f32" else (1e-10, 0.0)
    strict, loose = G.compare_argmin(best, cyc, ref, tol, 1e-6, btol)
    assert strict > 0
    # status: none-feasible exactly where the oracle has no candidate
    assert np.array_equal((status & klr.Q_NONE_FEASIBLE) != 0, ref["best"] < 0)
    # launch parameters: (ceil(N/b0), ceil(N/b1), 1, b0, b1, 1) or 3D
    cfg = klr.enumerate_configs(nv - 1)
    for r in range(0, len(best), max(1, len(best) // 50)):
        if best[r] < 0:
            assert np.all(launch[r] == 0)
            continue
        b = cfg[best[r]]
        N = int(q.sizes[r])
        g = [-(-N // int(b[i])) if i < nv - 1 else 1 for i in range(3)]
        assert list(launch[r]) == g + [int(v) for v in b]


def test_argmin_degree3_near_ties_match_oracle(klr, ctx):
    """Degree-3 programs put more queries within the FP32 window of a tie
    (among them, all four best shapes tied: the whole sweep redone in FP64).
    The usual bars hold, and every query re-decided in FP64 gets the oracle's
    choice wherever the oracle's margin is above 1e-9 (FP64 against FP64)."""
    gt = G.make_program(19, 96, degree=3)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(96, W.log_spaced_sizes(64))
    best, cyc, margin, status, launch = _run(klr, ctx, gt, coef, q.offsets, q.sizes, klr.F32, False)
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    table = ref["cycles"].reshape(len(q.sizes), -1)
    bnd = ref["boundary"].reshape(len(q.sizes), -1)
    ref = dict(ref, cycles=table, boundary=bnd)
    strict, loose = G.compare_argmin(best, cyc, ref, 1e-4, 1e-6, 1e-5)
    assert strict > 0
    tie = np.nonzero((status & klr.Q_TIE_RESOLVED) != 0)[0]
    assert len(tie) > 0
    checked = near = 0
    for r in tie:
        row = np.where(np.isfinite(table[r]), table[r], np.inf)
        order = np.argsort(row, kind="stable")
        bv = row[order[0]]
        m = (row[order[1]] - bv) / bv
        if m > 1e-9 and bnd[r, order[0]] > 1e-9:
            checked += 1
            assert best[r] == order[0], (r, best[r], order[0], m)
            assert abs(cyc[r] - bv) <= 1e-6 * bv
        elif m <= 1e-9 and bnd[r, best[r]] > 1e-9:
            # a tie in FP64 too: the choice must be one of the oracle's
            # minima (to FP64 rounding), not merely some configuration
            near += 1
            assert row[best[r]] <= bv * (1 + 1e-9), (r, best[r], row[best[r]], bv)
    assert checked > 0


def test_all_infeasible_and_empty_kernels(klr, ctx):
    gt = G.make_program(9, 3)
    gt.regs[:] = np.array([4096, 32, 64], dtype=np.int32)   # kernel 0: no block fits
    coef = gt.coef.astype(np.float32)
    # kernel 1 has no queries
    q_offsets = np.array([0, 4, 4, 7], dtype=np.int64)
    q_sizes = np.array([1024, 4096, 1 << 20, 64, 1 << 16, 300, 7], dtype=np.int64)
    best, cyc, margin, status, launch = _run(klr, ctx, gt, coef, q_offsets, q_sizes, klr.F32, False)
    assert np.all(best[:4] == -1) and np.all(np.isinf(cyc[:4]))
    assert np.all(status[:4] & klr.Q_NONE_FEASIBLE)
    ref = G.oracle_choose(coef, gt, q_offsets, q_sizes)
    assert np.array_equal(best, ref["best"])


def test_bad_arguments_return_einval(klr, ctx):
    gt = G.make_program(3, 1)
    ct = torch.tensor(gt.coef.astype(np.float32)).cuda()
    prog = G.gpu_program(klr, ct, gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    qo = torch.tensor([0, 2]).cuda()
    qn = torch.tensor([256, 512]).cuda()
    bad = klr.make_hw(dict(W.HARDWARE, n_sm=0))
    with pytest.raises(klr.KlrError) as e:
        ctx.argmin(prog, bad, cfg, qo, qn)
    assert e.value.status == klr.EINVAL
    with pytest.raises(klr.KlrError):
        ctx.eval(prog, hw, torch.zeros((300, 3), dtype=torch.int32).cuda(), qo, qn)


@pytest.mark.parametrize("kc,n_sizes", [(8, 64), (2, 8), (32, 16), (6, 64)])
def test_candidate_rerank_matches_oracle(klr, ctx, kc, n_sizes):
    """klr_argmin_candidates: per query the least-cycles meaningful shape among
    its candidates (ties to the lowest index), against the oracle's cycles
    table restricted to the same candidates.  The cases cover a kernel whose
    proposed shapes outnumber the specialised slots (8 x 64), all shapes
    specialised (2 x 8), whole warps per query (32) and a candidate count that
    is not a power of two (6: the block-per-kernel form)."""
    gt = G.make_program(6, 48)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(48, W.log_spaced_sizes(n_sizes))
    n_q = len(q.sizes)
    keys = W.stream_keys(41, (3,), np.arange(n_q, dtype=np.uint64))
    cand = (W.words(keys[:, None], np.arange(kc, dtype=np.uint64)[None, :]) % np.uint64(56))
    cand = cand.astype(np.int32) - 2          # -2..53: some skipped entries, some duplicates
    ct = torch.tensor(coef).cuda()
    prog = G.gpu_program(klr, ct, gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    best, cyc, st = klr.argmin_candidates(ctx, prog, hw, cfg, torch.tensor(q.offsets).cuda(),
                                          torch.tensor(q.sizes).cuda(), torch.tensor(cand).cuda())
    torch.cuda.synchronize()
    best, cyc, st = best.cpu().numpy(), cyc.cpu().numpy().astype(np.float64), st.cpu().numpy()
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    table = ref["cycles"].reshape(n_q, -1)
    bnd = ref["boundary"].reshape(n_q, -1)
    strict = 0
    for r in range(n_q):
        cs = sorted(set(int(c) for c in cand[r] if 0 <= c < 51))
        vals = [(table[r, c], c) for c in cs if np.isfinite(table[r, c])]
        if not vals:
            assert best[r] == -1 and (st[r] & klr.Q_NONE_FEASIBLE), r
            continue
        vals.sort()
        bv, bc = vals[0]
        margin = (vals[1][0] - bv) / bv if len(vals) > 1 else np.inf
        if margin > 1e-6 and bnd[r, bc] > 1e-5:
            strict += 1
            assert best[r] == bc, (r, best[r], bc, margin)
            assert abs(cyc[r] - bv) <= 1e-4 * bv
        elif (st[r] & klr.Q_TIE_RESOLVED) and margin > 1e-9 and bnd[r, bc] > 1e-9:
            # an FP32 near-tie re-decided in FP64: the oracle's choice
            assert best[r] == bc, (r, best[r], bc, margin)
            assert abs(cyc[r] - bv) <= 1e-6 * bv
        else:
            assert best[r] in cs and table[r, best[r]] <= bv * (1 + 4e-4)
    assert strict > 0.9 * n_q


@pytest.mark.parametrize("degree", [2, 3])
def test_candidate_rerank_equals_table_minimum(klr, ctx, degree):
    """The warp re-rank specialises the proposed shapes with the sweep's own
    sums, in the same order, and evaluates them with the same code: its cycles
    equal, bit for bit, the least entry of the sweep's FP32 cycles table over
    each query's candidates (ties to the lower shape index), and its choice is
    that entry's shape -- except where another candidate lies within the FP32
    error window of the least, which is re-decided in FP64 (flagged): there
    the choice is one of those near-tied candidates."""
    gt = G.make_program(7, 64, degree=degree)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(64, W.log_spaced_sizes(32))
    n_q, kc = len(q.sizes), 16
    keys = W.stream_keys(43, (degree,), np.arange(n_q, dtype=np.uint64))
    cand = (W.words(keys[:, None], np.arange(kc, dtype=np.uint64)[None, :]) % np.uint64(51))
    cand = cand.astype(np.int32)
    prog = G.gpu_program(klr, torch.tensor(coef).cuda(), gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    qo, qn = torch.tensor(q.offsets).cuda(), torch.tensor(q.sizes).cuda()
    table = ctx.eval(prog, hw, cfg, qo, qn, out_dtype=klr.F32)
    best, cyc, st = klr.argmin_candidates(ctx, prog, hw, cfg, qo, qn, torch.tensor(cand).cuda())
    torch.cuda.synchronize()
    table, best, cyc = table.cpu().numpy(), best.cpu().numpy(), cyc.cpu().numpy()
    tie = (st.cpu().numpy() & klr.Q_TIE_RESOLVED) != 0
    vals = np.take_along_axis(table, cand.astype(np.int64), axis=1)      # (n_q, kc)
    key = np.where(np.isfinite(vals), vals, np.inf)
    # least value, then least shape index
    order = np.lexsort((cand, key), axis=1)[:, 0]
    want_v = key[np.arange(n_q), order]
    want_c = np.where(np.isfinite(want_v), cand[np.arange(n_q), order], -1)
    # the FP32 window of the decision: another distinct candidate within it
    near = ((key.astype(np.float64) <= want_v.astype(np.float64)[:, None] * (1 + 5e-5))
            & (cand != want_c[:, None]))
    assert np.array_equal(tie, near.any(axis=1) & np.isfinite(want_v))
    ok = ~tie
    assert np.array_equal(best[ok], want_c[ok])
    fin = np.isfinite(want_v) & ok
    assert np.array_equal(cyc[fin], want_v[fin].astype(np.float32))
    for r in np.nonzero(tie)[0]:
        assert best[r] in cand[r] and key[r, list(cand[r]).index(best[r])] <= want_v[r] * (1 + 1e-4)
        assert abs(cyc[r] - want_v[r]) <= 1e-4 * want_v[r]
    assert fin.mean() > 0.5


@pytest.mark.parametrize("eps", [0.0, 0.02, 0.2])
def test_refined_choice_matches_oracle(klr, ctx, eps):
    """klr_argmin_refined on klr_eval's table against the oracle's refinement of
    its own FP64 table, wherever the decision is clear of the FP32/FP64
    difference (1e-4 relative) at the margin and between the finalists."""
    from oracle import program as oprog
    gt = G.make_program(6, 48)
    coef = gt.coef.astype(np.float32)
    q = W.queries_per_kernel(48, W.log_spaced_sizes(64))
    ct = torch.tensor(coef).cuda()
    prog = G.gpu_program(klr, ct, gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg_np = klr.enumerate_configs(2)
    cfg = torch.tensor(cfg_np).cuda()
    qo, qn = torch.tensor(q.offsets).cuda(), torch.tensor(q.sizes).cuda()
    table = ctx.eval(prog, hw, cfg, qo, qn, out_dtype=klr.F32)
    best, cyc, st = klr.argmin_refined(ctx, prog, hw, cfg, qo, qn, table, eps)
    torch.cuda.synchronize()
    best, cyc, st = best.cpu().numpy(), cyc.cpu().numpy(), st.cpu().numpy()
    tab = table.cpu().numpy().astype(np.float64)
    ref = G.oracle_choose(coef, gt, q.offsets, q.sizes)
    otab = ref["cycles"].reshape(len(q.sizes), -1)
    configs = [tuple(int(v) for v in c) for c in cfg_np[:, :2]]
    strict = 0
    for k in range(48):
        _, Wk = oprog.kernel_occupancy(int(gt.regs[k]), int(gt.smem[k]), configs, W.HARDWARE)
        for r in range(int(q.offsets[k]), int(q.offsets[k + 1])):
            row = otab[r]
            want = oprog.refine(row[None, :], Wk, eps)[0]
            fin = np.isfinite(row)
            if want < 0:
                assert best[r] == -1 and (st[r] & klr.Q_NONE_FEASIBLE)
                continue
            # every GPU choice is valid on the GPU's own table
            gfin = np.isfinite(tab[r])
            glo = tab[r][gfin].min()
            assert tab[r, best[r]] <= glo * (1 + eps) and cyc[r] == np.float32(tab[r, best[r]])
            near = [c for c in range(len(row)) if fin[c] and row[c] <= row[fin].min() * (1 + eps)]
            lo = row[fin].min()
            thr = lo * (1 + eps)
            # entries that FP32 rounding could move across the margin (the
            # least itself is always inside)
            clear_margin = not np.any(fin & (np.abs(row - thr) <= 1e-4 * thr) & (row > lo))
            others = [c for c in near if c != want]
            clear_pick = all(Wk[c] < Wk[want] or abs(row[c] - row[want]) > 1e-4 * row[want]
                             for c in others)
            if clear_margin and clear_pick:
                strict += 1
                assert best[r] == want, (r, best[r], want)
                if np.sum(fin & (row <= lo * (1 + 1e-4))) == 1:      # unambiguous least cycles
                    first = int(np.argmin(np.where(fin, row, np.inf)))
                    assert bool(st[r] & klr.Q_REFINED) == (want != first)
    assert strict > 0.8 * len(q.sizes)


@pytest.mark.parametrize("seed,nv,degree", [(31, 3, 2), (32, 3, 1), (33, 4, 3), (34, 4, 2)])
def test_fp64_latency_mode_equals_the_kernel_sweep(klr, ctx, seed, nv, degree):
    """An FP64 argmin of at most 1024 queries runs one block per query; a
    larger one runs a block per kernel.  The same queries asked both ways (a batch of
    1200, then slices of it) give bitwise equal outputs: index, cycles,
    margin, status bits and launch geometry.  Kernel 1 has no queries, kernel
    0 fits no block, and the sizes include N below every shape."""
    nk = 12
    gt = G.make_program(seed, nk, n_vars=nv, degree=degree)
    gt.regs[0] = 4096
    coef = gt.coef.astype(np.float64)
    rng = np.random.default_rng(seed)
    per = np.full(nk, 1200 // (nk - 1), dtype=np.int64)
    per[1] = 0
    per[-1] += 1200 - per.sum()
    q_off = np.concatenate([[0], np.cumsum(per)]).astype(np.int64)
    sizes = np.exp2(rng.uniform(0, 26, size=1200)).astype(np.int64)
    sizes[::97] = 1
    sizes[5::89] = 7
    full = _run(klr, ctx, gt, coef, q_off, sizes, klr.F64, False)
    for lo_q, hi_q in ((0, 1024), (300, 301), (513, 1200)):
        # the slice's queries, with each kernel's offsets clipped to it
        off = np.clip(q_off, lo_q, hi_q) - lo_q
        part = _run(klr, ctx, gt, coef, off, sizes[lo_q:hi_q], klr.F64, False)
        for a, b in zip(full, part):
            assert np.array_equal(a[lo_q:hi_q].view(np.uint8), b.view(np.uint8)), (lo_q, hi_q)
    best, cyc, status = full[0], full[1], full[3]
    assert np.all(best[:q_off[1]] == -1) and np.all(status[:q_off[1]] & klr.Q_NONE_FEASIBLE)
    assert np.any(best >= 0) and np.all(np.isfinite(cyc[best >= 0]))


def test_page_locked_host_queries_give_the_same_choices(klr, ctx):
    """klr_argmin's queries may be page-locked host memory, read in place:
    the outputs equal those of the same queries in device memory."""
    gt = G.make_program(35, 16)
    ct = torch.tensor(gt.coef.astype(np.float32)).cuda()
    prog = G.gpu_program(klr, ct, gt, torch)
    hw = klr.make_hw(W.HARDWARE)
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    q = W.queries_per_kernel(16, W.log_spaced_sizes(64))
    qo_h = torch.from_numpy(q.offsets).pin_memory()
    qn_h = torch.from_numpy(q.sizes).pin_memory()
    a = ctx.argmin(prog, hw, cfg, qo_h, qn_h)
    b = ctx.argmin(prog, hw, cfg, qo_h.cuda(), qn_h.cuda())
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert x.is_cuda and torch.equal(x, y)
