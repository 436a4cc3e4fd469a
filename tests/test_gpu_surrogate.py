"""GPU tests of the learned proposer (the surrogate network's BF16 training and
inference kernels) against the FP64 oracle, and of what it gains.

Gradient tolerance, derived from the arithmetic: the kernels use BF16 operands
(unit roundoff 2^-9) with FP32 accumulation.  The oracle is given the same
BF16-rounded weights, coefficients and features, so the remaining difference is
the BF16 rounding of the activations and backward signals between layers (a
few roundings per path, each 2^-9): relative L2 error per parameter tensor
within 4e-2, and the loss within 2e-2.
"""
import numpy as np
import pytest

import workloads as W
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

HW_FEAT = np.ones(7, dtype=np.float32)


@pytest.fixture(scope="module")
def klr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as k
    return k


@pytest.fixture(scope="module")
def ctx(klr):
    return klr.Context(0)


def _bf16(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).bfloat16().double().numpy()


def _init(klr, n_coef, seed, n_out=0):
    from paper_1911_02373_gb300 import proposer
    n = klr.mlp_param_count(n_coef, n_out)
    keys = W.stream_keys(seed, (77,), np.arange(1, dtype=np.uint64))
    z = W.normal(keys[0], np.arange(n, dtype=np.uint64))
    return proposer.init_params(n_coef, z, n_out)


def test_gradients_match_oracle(klr, ctx):
    gt = W.ground_truth(31, 12, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    coef = gt.coef.reshape(12, n_coef).astype(np.float32)
    rng = np.random.default_rng(0)
    n = 300
    kern = rng.integers(0, 12, n).astype(np.int32)
    N = (2 ** rng.uniform(8, 23, n)).astype(np.int64)
    cfg = klr.enumerate_configs(2)
    ci = rng.integers(0, len(cfg), n).astype(np.int32)
    target = rng.standard_normal(n).astype(np.float32)
    init = _init(klr, n_coef, 5)
    sur = klr.Surrogate(ctx, n_coef, init, HW_FEAT)
    grads = torch.zeros(init.size, dtype=torch.float32, device="cuda")
    t = lambda a: torch.tensor(a).cuda()
    loss = sur.train_step(t(coef), t(cfg), t(kern), t(N), t(ci), t(target), 0.0, 0.0, False,
                          grads=grads)
    torch.cuda.synchronize()
    g_gpu = grads.cpu().numpy().astype(np.float64)
    # oracle with the kernels' BF16 inputs and weights (biases stay FP32)
    p = omlp.unpack(init.astype(np.float64), n_coef)
    for name in ("E", "W1", "W2", "W3", "W4"):
        p[name] = _bf16(p[name])
    feat = _bf16(omlp.features(N, cfg[ci], HW_FEAT))
    loss_ref, g_ref = omlp.loss_and_grads(p, feat, _bf16(coef[kern]), target.astype(np.float64))
    assert abs(float(loss.item()) - loss_ref) <= 2e-2 * abs(loss_ref)
    gg = omlp.unpack(g_gpu, n_coef)
    for name, _ in omlp.shapes(n_coef):
        ref = np.asarray(g_ref[name], dtype=np.float64).reshape(-1)
        got = np.asarray(gg[name]).reshape(-1)
        rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert rel <= 4e-2, (name, rel)
    # predictions: same bound on the forward pass alone
    pred = sur.predict(t(coef), t(cfg), t(kern), t(N), t(ci))
    pr_ref, _ = omlp.forward(p, feat, _bf16(coef[kern]))
    got = pred.cpu().numpy()
    assert np.linalg.norm(got - pr_ref) <= 4e-2 * np.linalg.norm(pr_ref)


def test_head_gradients_match_oracle(klr, ctx):
    """The per-query form: 51 outputs per (kernel, N) row, masked targets."""
    gt = W.ground_truth(35, 10, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    coef = gt.coef.reshape(10, n_coef).astype(np.float32)
    rng = np.random.default_rng(5)
    n, n_out = 260, 51
    kern = rng.integers(0, 10, n).astype(np.int32)
    N = (2 ** rng.uniform(8, 23, n)).astype(np.int64)
    target = rng.standard_normal((n, n_out)).astype(np.float32)
    target[rng.random((n, n_out)) < 0.25] = np.nan
    cfg = klr.enumerate_configs(2)
    init = _init(klr, n_coef, 9, n_out)
    sur = klr.Surrogate(ctx, n_coef, init, HW_FEAT, n_out=n_out)
    grads = torch.zeros(init.size, dtype=torch.float32, device="cuda")
    t = lambda a: torch.tensor(a).cuda()
    loss = sur.train_step(t(coef), t(cfg), t(kern), t(N), None, t(target), 0.0, 0.0, False,
                          grads=grads)
    torch.cuda.synchronize()
    g_gpu = grads.cpu().numpy().astype(np.float64)
    p = omlp.unpack(init.astype(np.float64), n_coef, n_out)
    for name in ("E", "W1", "W2", "W3", "W4"):
        p[name] = _bf16(p[name])
    feat = _bf16(omlp.features(N, None, HW_FEAT))
    loss_ref, g_ref = omlp.loss_and_grads(p, feat, _bf16(coef[kern]), target.astype(np.float64))
    assert abs(float(loss.item()) - loss_ref) <= 2e-2 * abs(loss_ref)
    gg = omlp.unpack(g_gpu, n_coef, n_out)
    for name, _ in omlp.shapes(n_coef, n_out):
        ref = np.asarray(g_ref[name], dtype=np.float64).reshape(-1)
        got = np.asarray(gg[name]).reshape(-1)
        rel = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert rel <= 4e-2, (name, rel)
    pred = sur.predict(t(coef), t(cfg), t(kern), t(N), None)
    pr_ref, _ = omlp.forward(p, feat, _bf16(coef[kern]), per_query=True)
    got = pred.cpu().numpy()
    assert got.shape == (n, n_out)
    assert np.linalg.norm(got - pr_ref) <= 4e-2 * np.linalg.norm(pr_ref)


def test_query_targets_are_centred_log2_cycles(klr, ctx):
    rng = np.random.default_rng(6)
    cyc = (2.0 ** rng.uniform(5, 30, (300, 51))).astype(np.float32)
    cyc[rng.random((300, 51)) < 0.3] = np.inf
    cyc[7, :] = np.inf                       # a query with no meaningful shape
    got = klr.query_targets(torch.tensor(cyc).cuda()).cpu().numpy()
    lg = np.log2(cyc.astype(np.float64))
    fin = np.isfinite(lg)
    mean = np.array([lg[r][fin[r]].mean() if fin[r].any() else 0.0 for r in range(300)])
    want = np.where(fin, lg - mean[:, None], np.nan)
    assert np.array_equal(np.isnan(got), ~fin)
    assert np.allclose(got[fin], want[fin], rtol=0, atol=2e-5)


def test_adamw_step_matches_oracle(klr, ctx):
    gt = W.ground_truth(32, 4, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    coef = gt.coef.reshape(4, n_coef).astype(np.float32)
    init = _init(klr, n_coef, 6)
    sur = klr.Surrogate(ctx, n_coef, init, HW_FEAT)
    rng = np.random.default_rng(1)
    n = 64
    cfg = klr.enumerate_configs(2)
    t = lambda a: torch.tensor(a).cuda()
    args = (t(coef), t(cfg), t(rng.integers(0, 4, n).astype(np.int32)),
            t((2 ** rng.uniform(8, 23, n)).astype(np.int64)),
            t(rng.integers(0, 51, n).astype(np.int32)), t(rng.standard_normal(n).astype(np.float32)))
    grads = torch.zeros(init.size, dtype=torch.float32, device="cuda")
    sur.train_step(*args, 1e-3, 0.01, True, grads=grads)
    torch.cuda.synchronize()
    g = grads.cpu().numpy().astype(np.float64)
    want, m, v = omlp.adamw(init.astype(np.float64), g, np.zeros_like(g), np.zeros_like(g), 1,
                            lr=1e-3, wd=0.01)
    assert np.allclose(sur.params.cpu().numpy(), want, rtol=0, atol=2e-6)
    assert np.allclose(sur.m.cpu().numpy(), m, rtol=1e-5, atol=1e-9)


def test_training_is_bitwise_reproducible(klr, ctx):
    """Every sum over rows in a training step (split-K slices, bias gradients,
    the loss) is added in a fixed order, so two runs from the same start give
    identical parameters and moments."""
    gt = W.ground_truth(34, 6, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    coef = torch.tensor(gt.coef.reshape(6, n_coef).astype(np.float32)).cuda()
    cfg = torch.tensor(klr.enumerate_configs(2)).cuda()
    rng = np.random.default_rng(2)
    n = 5000                                   # several split-K slices and reduction blocks
    t = lambda a: torch.tensor(a).cuda()
    batches = [(t(rng.integers(0, 6, n).astype(np.int32)),
                t((2 ** rng.uniform(8, 23, n)).astype(np.int64)),
                t(rng.integers(0, 51, n).astype(np.int32)),
                t(rng.standard_normal(n).astype(np.float32))) for _ in range(3)]
    init = _init(klr, n_coef, 8)
    runs = []
    for _ in range(2):
        sur = klr.Surrogate(ctx, n_coef, init, HW_FEAT)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        for b in batches:
            sur.train_step(coef, cfg, *b, 1e-3, 0.01, True, loss)
        torch.cuda.synchronize()
        runs.append((sur.params.cpu().numpy(), sur.m.cpu().numpy(), sur.v.cpu().numpy(),
                     loss.cpu().numpy()))
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_trained_proposer_beats_random_candidates(klr, ctx):
    from paper_1911_02373_gb300 import proposer
    nk = 160
    gt = W.ground_truth(33, nk, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    coef_np = gt.coef.astype(np.float32)
    t = lambda a: torch.tensor(a).cuda()
    coef3 = t(coef_np)
    coef = coef3.reshape(nk, n_coef)
    regs, smem = t(gt.regs), t(gt.smem)
    cfg = t(klr.enumerate_configs(2))
    hw = klr.make_hw(W.HARDWARE)
    prog = klr.Context.program(coef3, regs, smem, n_vars=3, degree=3, n_scale_log2=23,
                               b_scale_log2=10, metric_lo=W.METRIC_LO, metric_scale=W.METRIC_SCALE)
    # training rows: every (size, shape) of 64 log-spaced sizes, meaningful ones kept
    sizes = W.log_spaced_sizes(64)
    q = W.queries_per_kernel(nk, sizes)
    qo, qn = t(q.offsets), t(q.sizes)
    nq = len(q.sizes)
    rq = torch.arange(nq, device="cuda").repeat_interleave(51)
    rc = torch.arange(51, device="cuda").repeat(nq)
    y = proposer.table_targets(ctx, prog, hw, cfg, qo, qn, rq, rc)
    keep = torch.isfinite(y)
    rq, rc, y = rq[keep], rc[keep], y[keep]
    target = y.float().contiguous()
    kern = (rq // 64).int().contiguous()
    N = qn[rq].contiguous()
    ci = rc.int().contiguous()
    sur = klr.Surrogate(ctx, n_coef, _init(klr, n_coef, 7), HW_FEAT)
    n = kern.numel()
    keys = W.stream_keys(8, (78,), np.arange(40, dtype=np.uint64))
    order = lambda ep: t(np.argsort(W.words(keys[ep], np.arange(n, dtype=np.uint64)), kind="stable"))
    losses = proposer.train(sur, coef, cfg, kern, N, ci, target, batch=4096, epochs=16, lr=2e-3,
                            order=order, log_every=20)
    assert losses[-1] < 0.25 * losses[0], losses
    # evaluation queries: 16 sizes per kernel not on the training grid
    ev = np.unique(np.floor(np.exp2(np.linspace(8.3, 22.7, 16))).astype(np.int64))
    qe = W.queries_per_kernel(nk, ev)
    qeo, qen = t(qe.offsets), t(qe.sizes)
    best, cyc, mg, st, _ = ctx.argmin(prog, hw, cfg, qeo, qen, out_dtype=klr.F32)
    sb, sc, sst, cand = proposer.propose_and_rerank(ctx, sur, prog, hw, coef, regs, smem, cfg, qeo,
                                                    qen, 8)
    # random 8 candidates per query, re-ranked the same way
    kr = W.stream_keys(9, (79,), np.arange(len(qe.sizes), dtype=np.uint64))
    rnd = (W.words(kr[:, None], np.arange(8, dtype=np.uint64)[None, :]) % np.uint64(51)).astype(np.int32)
    rb, rcyc, _ = klr.argmin_candidates(ctx, prog, hw, cfg, qeo, qen, t(rnd))
    torch.cuda.synchronize()
    c_best = cyc.cpu().numpy().astype(np.float64)
    ok = np.isfinite(c_best)
    reg_s = sc.cpu().numpy()[ok] / c_best[ok] - 1
    reg_r = rcyc.cpu().numpy()[ok] / c_best[ok] - 1
    reg_r = np.where(np.isfinite(reg_r), reg_r, 10.0)
    assert np.all(reg_s >= -1e-5)
    assert np.mean(reg_s) < 0.5 * np.mean(reg_r), (np.mean(reg_s), np.mean(reg_r))
    assert np.median(reg_s) < 0.05


def test_trained_head_proposer_beats_random_candidates(klr, ctx):
    """The per-query form trained on the same programs: one row per (kernel, N)
    with 51 masked targets."""
    from paper_1911_02373_gb300 import proposer
    nk = 160
    gt = W.ground_truth(33, nk, 3, 3, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    t = lambda a: torch.tensor(a).cuda()
    coef3 = t(gt.coef.astype(np.float32))
    coef = coef3.reshape(nk, n_coef)
    regs, smem = t(gt.regs), t(gt.smem)
    cfg = t(klr.enumerate_configs(2))
    hw = klr.make_hw(W.HARDWARE)
    prog = klr.Context.program(coef3, regs, smem, n_vars=3, degree=3, n_scale_log2=23,
                               b_scale_log2=10, metric_lo=W.METRIC_LO, metric_scale=W.METRIC_SCALE)
    sizes = W.log_spaced_sizes(64)
    q = W.queries_per_kernel(nk, sizes)
    qo, qn = t(q.offsets), t(q.sizes)
    target = proposer.query_table(ctx, prog, hw, cfg, qo, qn)
    keep = torch.isfinite(target).any(dim=1)
    rows = torch.nonzero(keep)[:, 0]
    kern = (rows // 64).int().contiguous()
    N = qn[rows].contiguous()
    target = target[rows].contiguous()
    sur = klr.Surrogate(ctx, n_coef, _init(klr, n_coef, 10, 51), HW_FEAT, n_out=51)
    n = kern.numel()
    keys = W.stream_keys(8, (80,), np.arange(200, dtype=np.uint64))
    order = lambda ep: t(np.argsort(W.words(keys[ep], np.arange(n, dtype=np.uint64)), kind="stable"))
    losses = proposer.train(sur, coef, cfg, kern, N, None, target, batch=512, epochs=120, lr=2e-3,
                            order=order, log_every=20)
    assert losses[-1] < 0.25 * losses[0], losses
    ev = np.unique(np.floor(np.exp2(np.linspace(8.3, 22.7, 16))).astype(np.int64))
    qe = W.queries_per_kernel(nk, ev)
    qeo, qen = t(qe.offsets), t(qe.sizes)
    best, cyc, mg, st, _ = ctx.argmin(prog, hw, cfg, qeo, qen, out_dtype=klr.F32)
    sb, sc, sst, cand = proposer.propose_and_rerank(ctx, sur, prog, hw, coef, regs, smem, cfg, qeo,
                                                    qen, 8)
    kr = W.stream_keys(9, (79,), np.arange(len(qe.sizes), dtype=np.uint64))
    rnd = (W.words(kr[:, None], np.arange(8, dtype=np.uint64)[None, :]) % np.uint64(51)).astype(np.int32)
    rb, rcyc, _ = klr.argmin_candidates(ctx, prog, hw, cfg, qeo, qen, t(rnd))
    torch.cuda.synchronize()
    c_best = cyc.cpu().numpy().astype(np.float64)
    ok = np.isfinite(c_best)
    reg_s = sc.cpu().numpy()[ok] / c_best[ok] - 1
    reg_r = rcyc.cpu().numpy()[ok] / c_best[ok] - 1
    reg_r = np.where(np.isfinite(reg_r), reg_r, 10.0)
    assert np.all(reg_s >= -1e-5)
    assert np.mean(reg_s) < 0.5 * np.mean(reg_r), (np.mean(reg_s), np.mean(reg_r))
    assert np.median(reg_s) < 0.05


@pytest.mark.parametrize("dims,k", [(2, 8), (2, 16), (3, 5)])
def test_proposal_is_topk_of_predictions(klr, ctx, dims, k):
    """klr_propose's fused top-k against the network's own outputs: for every
    query, the k meaningful shapes (B_active > 0 by Fig. 1, every block side
    <= N) of least prediction, ties to the lower shape index, -1 past the
    meaningful ones.  The proposal builds its input rows inside the kernel and
    never writes the outputs; klr_mlp_predict writes them from the same
    network, so the two agree exactly.  60,000 queries: several 128-row tiles
    per CTA and a ragged last tile; 251 shapes (3D) put four 16-column chunks
    in every column group."""
    from oracle import occupancy as oocc
    nk, per = 500, 120
    gt = W.ground_truth(51, nk, 3, 2, 8, 23, 10)
    n_coef = 8 * gt.coef.shape[-1]
    cfg_np = klr.enumerate_configs(dims)
    n_cfg = len(cfg_np)
    t = lambda a: torch.tensor(a).cuda()
    coef = t(gt.coef.astype(np.float32)).reshape(nk, n_coef)
    regs, smem, cfg = t(gt.regs), t(gt.smem), t(cfg_np)
    hw = klr.make_hw(W.HARDWARE)
    q = W.queries_per_kernel(nk, W.log_spaced_sizes(per))
    qo, qn = t(q.offsets), t(q.sizes)
    sur = klr.Surrogate(ctx, n_coef, _init(klr, n_coef, 12 + dims, n_cfg), HW_FEAT, n_out=n_cfg)
    cand = sur.propose(coef, regs, smem, hw, cfg, qo, qn, k)
    kern = t(np.repeat(np.arange(nk, dtype=np.int32), per))
    pred = sur.predict(coef, cfg, kern, qn, None)
    torch.cuda.synchronize()
    cand, pred = cand.cpu().numpy(), pred.cpu().numpy()
    T = np.prod(cfg_np.astype(np.int64), axis=1)
    occ = np.array([[oocc.active_blocks(int(T[c]), int(gt.regs[i]), int(gt.smem[i]), W.HARDWARE) > 0
                     for c in range(n_cfg)] for i in range(nk)])
    bmax = cfg_np.max(axis=1)
    mask = occ[np.repeat(np.arange(nk), per)] & (bmax[None, :] <= q.sizes[:, None])
    val = np.where(mask & np.isfinite(pred), pred, np.inf)
    order = np.argsort(val, axis=1, kind="stable")[:, :k]      # value, then index
    want = np.where(np.isfinite(np.take_along_axis(val, order, axis=1)), order, -1)
    assert np.all(mask.sum(axis=1) > 0)
    assert np.array_equal(cand, want), np.argwhere(cand != want)[:5]
