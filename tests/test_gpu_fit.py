"""GPU parity of the batched rational fit (F1-F4) against the FP64 oracle,
through the C ABI.

Tolerance, derived from the arithmetic: the library solves the eigenproblem of
the Gram matrix G of the equilibrated design matrix, accumulated with unit
roundoff eps_acc (2^-53 for FP64, about 2^-44 for DF32 pairs, 2^-24 for FP32).
A perturbation E of G moves the null vector by about |E| / gap, with
|E| <= c u eps_acc |G| and gap = (sigma_{u-1}^2 - sigma_u^2) / sigma_1^2 the
relative eigen-gap the oracle reports.  Each FP64 refinement pass over the
samples multiplies the error by about eps_acc kappa^2 again, down to the
FP64 floor of the SVD itself (eps_64 times kappa).  The coefficient bound used
below is  64 u eps_acc / gap  (no refinement) or that bound squared with the
floor, and predictions on the evaluation grid follow the coefficients.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import rational

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = {"fp64": 2.0 ** -53, "df32": 2.0 ** -44, "fp32": 2.0 ** -24}


@pytest.fixture(scope="module")
def klr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1911_02373_gb300 as k
    return k


@pytest.fixture(scope="module")
def ctx(klr):
    return klr.Context(0)


def gpu_fit(klr, ctx, fb, precision, refine=0, coef_dtype=None):
    off = torch.tensor(fb.offsets).cuda()
    x = torch.tensor(np.ascontiguousarray(fb.x)).cuda()
    y = torch.tensor(fb.y).cuda()
    coef, status, diag = ctx.fit(off, x, y, n_vars=fb.n_vars, degree=fb.degree,
                                 n_scale_log2=fb.n_scale_log2, b_scale_log2=fb.b_scale_log2,
                                 precision=precision, refine_iters=refine,
                                 coef_dtype=klr.F64 if coef_dtype is None else coef_dtype)
    torch.cuda.synchronize()
    return coef.cpu().numpy().astype(np.float64), status.cpu().numpy(), diag.cpu().numpy()


def bound(mode, u, gap, refine):
    b = 64.0 * u * EPS[mode] / gap
    for _ in range(refine):
        b = b * min(1.0, 64.0 * u * EPS[mode] / gap)
    return max(b, 1e-11)


def check(fb, coef, status, mode, refine, ref=None):
    oc, ost, od = ref if ref is not None else rational.fit_batch(
        fb.offsets, fb.x.astype(np.float64), fb.y.astype(np.float64), fb.n_vars, fb.degree,
        fb.n_scale_log2, fb.b_scale_log2)
    u = coef.shape[1]
    errs = []
    for f in range(len(oc)):
        if ost[f] & rational.FIT_RANK_DEFICIENT:
            continue
        assert (int(status[f]) & ~8) == int(ost[f]), (f, status[f], ost[f])
        gap = max(od[f][1] ** 2 - od[f][0] ** 2, 1e-300)
        err = float(np.max(np.abs(coef[f] - oc[f])))
        errs.append(err)
        assert err <= bound(mode, u, gap, refine), (f, err, bound(mode, u, gap, refine), gap)
    return max(errs) if errs else 0.0


def test_single_kernel_fp64_exact_recovery(klr, ctx):
    fb = W.fit_batch(21, 1, 200, dtype=np.float64)
    for refine in (0, 1):
        coef, st, diag = gpu_fit(klr, ctx, fb, klr.FIT_FP64, refine)
        assert np.all(st == 0)
        m = coef.shape[1] // 2
        truth = fb.truth.coef[0] / np.linalg.norm(fb.truth.coef[0], axis=1, keepdims=True)
        truth *= np.sign(truth[:, m:m + 1])
        assert np.max(np.abs(coef - truth)) <= (1e-8 if refine == 0 else 1e-10)
        check(fb, coef, st, "fp64", refine)
        assert np.all(diag[:, 3] == refine)


def test_df32_noiseless_float32_samples(klr, ctx):
    fb = W.fit_batch(22, 4, 300, dtype=np.float32)
    coef, st, _ = gpu_fit(klr, ctx, fb, klr.FIT_DF32, 0)
    assert np.all(st == 0)
    check(fb, coef, st, "df32", 0)
    coef1, st1, _ = gpu_fit(klr, ctx, fb, klr.FIT_DF32, 1)
    check(fb, coef1, st1, "df32", 1)


@pytest.mark.parametrize("mode", ["df32", "fp64"])
def test_batched_noisy_ragged(klr, ctx, mode):
    fb = W.fit_batch(23, 24, (50, 2000), noise=0.01, dtype=np.float32)
    prec = klr.FIT_DF32 if mode == "df32" else klr.FIT_FP64
    coef, st, _ = gpu_fit(klr, ctx, fb, prec, 0, coef_dtype=klr.F32)
    # coefficients are returned in FP32: add its rounding to the bound
    ref = rational.fit_batch(fb.offsets, fb.x.astype(np.float64), fb.y.astype(np.float64),
                             3, 2, 23, 10)
    oc, ost, od = ref
    for f in range(len(oc)):
        gap = max(od[f][1] ** 2 - od[f][0] ** 2, 1e-300)
        err = np.max(np.abs(coef[f] - oc[f]))
        assert err <= bound(mode, 20, gap, 0) + 2.0 ** -24, (f, err, gap)


def test_df32_binned_and_per_sample_fits_in_one_batch(klr, ctx):
    """DF32 degree-2 fits go through per-cell sums when every sample is a
    power of two inside the 16 octaves of N below the N scale and has one of
    the 51 block shapes of 32..1024 threads; any other fit is left to the
    per-sample moments kernel.  One batch with both kinds, and the statuses
    of an empty fit and a fit with a NaN sample."""
    from types import SimpleNamespace
    fb = W.fit_batch(25, 3, (50, 600), noise=0.01, dtype=np.float32)
    xs = [fb.x[:, fb.offsets[f]:fb.offsets[f + 1]].copy() for f in range(fb.n_fits)]
    ys = [fb.y[fb.offsets[f]:fb.offsets[f + 1]].copy() for f in range(fb.n_fits)]
    xs[1][0, 0] = 2.0 ** 7                 # one octave below the window
    xs[3][1:, 0] = (4.0, 4.0)              # a 16-thread block shape
    xs[5][0, 0] = 2.0 ** 24                # above the N scale
    ys[7][3] = np.nan                      # non-finite sample
    xs[9], ys[9] = xs[9][:, :0], ys[9][:0]  # empty fit
    xs[11][0, -1] = 2.0 ** 8               # edge of the window (t = 15): binned
    xs[11][1:, -1] = (1024.0, 1.0)         # edge shape: binned
    off = np.concatenate([[0], np.cumsum([len(v) for v in ys])]).astype(np.int64)
    b = SimpleNamespace(offsets=off, x=np.concatenate(xs, axis=1).astype(np.float32),
                        y=np.concatenate(ys).astype(np.float32), n_vars=3, degree=2,
                        n_scale_log2=23, b_scale_log2=10)
    coef, st, _ = gpu_fit(klr, ctx, b, klr.FIT_DF32, 0)
    assert st[9] == rational.FIT_EMPTY and st[7] == rational.FIT_NONFINITE
    assert np.all(coef[9] == 0) and np.all(coef[7] == 0)
    check(b, coef, st, "df32", 0)
    # the same batch twice: the binned path is deterministic
    coef2, st2, _ = gpu_fit(klr, ctx, b, klr.FIT_DF32, 0)
    assert np.array_equal(coef, coef2) and np.array_equal(st, st2)


def test_df32_per_sample_fits_scattered_over_a_large_batch(klr, ctx):
    """After the binned kernel the per-sample moments kernel runs on one
    resident wave of blocks (4 per SM of 4 warps) whose warps step over the
    fits, testing 32 of their fits per flag load; in a batch of 96,000 fits
    (more than 32 times that wave's warps) every 7th fit has an N below the
    binned window.  Those fits equal, bit for bit, the same fits fitted as a
    batch of their own, which the oracle checks."""
    from types import SimpleNamespace
    fb = W.fit_batch(28, 12000, (48, 64), noise=0.01, dtype=np.float32)
    x = np.ascontiguousarray(fb.x).copy()
    pick = np.arange(3, fb.n_fits, 7)
    x[0, fb.offsets[pick]] = 2.0 ** 7      # one octave below the window
    big = SimpleNamespace(offsets=fb.offsets, x=x, y=fb.y, n_vars=3, degree=2,
                          n_scale_log2=23, b_scale_log2=10)
    coef, st, _ = gpu_fit(klr, ctx, big, klr.FIT_DF32, 0)
    idx = np.concatenate([np.arange(fb.offsets[f], fb.offsets[f + 1]) for f in pick])
    off = np.concatenate([[0], np.cumsum(np.diff(fb.offsets)[pick])]).astype(np.int64)
    sub = SimpleNamespace(offsets=off, x=np.ascontiguousarray(x[:, idx]), y=fb.y[idx],
                          n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10)
    coef_s, st_s, _ = gpu_fit(klr, ctx, sub, klr.FIT_DF32, 0)
    assert np.array_equal(coef[pick], coef_s) and np.array_equal(st[pick], st_s)
    check(sub, coef_s, st_s, "df32", 0)
    # the fits the binned kernel took are untouched by the fallback launch
    coef_b, st_b, _ = gpu_fit(klr, ctx, fb, klr.FIT_DF32, 0)
    keep = np.setdiff1d(np.arange(fb.n_fits), pick)
    assert np.array_equal(coef[keep], coef_b[keep]) and np.array_equal(st[keep], st_b[keep])


def test_df32_fits_beyond_the_binned_sample_limit(klr, ctx):
    """Fits with more samples than a 16-bit cell count holds (65,535) take
    the per-sample moments kernel; a batch mixing them with binned fits."""
    from types import SimpleNamespace
    big = W.fit_batch(26, 1, 70000, noise=0.01, dtype=np.float32)
    small = W.fit_batch(27, 1, 400, noise=0.01, dtype=np.float32)
    pick = [0, 3]                          # two big fits, then the small batch
    xs = [big.x[:, big.offsets[f]:big.offsets[f + 1]] for f in pick]
    ys = [big.y[big.offsets[f]:big.offsets[f + 1]] for f in pick]
    xs += [small.x[:, small.offsets[f]:small.offsets[f + 1]] for f in range(small.n_fits)]
    ys += [small.y[small.offsets[f]:small.offsets[f + 1]] for f in range(small.n_fits)]
    off = np.concatenate([[0], np.cumsum([len(v) for v in ys])]).astype(np.int64)
    b = SimpleNamespace(offsets=off, x=np.concatenate(xs, axis=1).astype(np.float32),
                        y=np.concatenate(ys).astype(np.float32), n_vars=3, degree=2,
                        n_scale_log2=23, b_scale_log2=10)
    coef, st, _ = gpu_fit(klr, ctx, b, klr.FIT_DF32, 0)
    check(b, coef, st, "df32", 0)


def test_exp8_samples_equal_float32_samples(klr, ctx):
    """KLR_EXP8 (uint8 base-2 logarithms of the coordinates) carries the same
    power-of-two samples in 7 bytes instead of 16: every output equals the
    FP32-input fit's bit for bit, the per-sample route included (a fit with
    an N outside the 16 binned octaves, one with a coordinate of 2^200, which
    is not finite, and an empty one)."""
    fb = W.fit_batch(28, 3, (50, 900), noise=0.01, dtype=np.float32)
    e = np.round(np.log2(fb.x.astype(np.float64))).astype(np.int64)
    assert np.array_equal(np.ldexp(1.0, e), fb.x)
    e[0, fb.offsets[2]] = 6                       # N = 64: per-sample route
    e[1, fb.offsets[5] + 1] = 200                 # 2^200: not finite
    x8 = e.astype(np.uint8)
    x32 = np.where(e <= 127, np.ldexp(1.0, np.minimum(e, 127)), np.inf).astype(np.float32)
    off = fb.offsets.copy()
    off[9:] = off[9:] - (off[9] - off[8])         # fit 8 empty
    n = int(off[-1])
    keep = np.r_[0:fb.offsets[8], fb.offsets[9]:fb.offsets[-1]]
    x8, x32, y = x8[:, keep], x32[:, keep], fb.y[keep]
    assert x8.shape[1] == n
    t = lambda a: torch.tensor(np.ascontiguousarray(a)).cuda()
    kw = dict(n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10, precision=klr.FIT_DF32,
              refine_iters=0, coef_dtype=klr.F32)
    c8, s8, d8 = ctx.fit(t(off), t(x8), t(y), **kw)
    c32, s32, d32 = ctx.fit(t(off), t(x32), t(y), **kw)
    torch.cuda.synchronize()
    assert torch.equal(c8, c32) and torch.equal(s8, s32) and torch.equal(d8, d32)
    st = s8.cpu().numpy()
    assert st[5] == rational.FIT_NONFINITE and st[8] == rational.FIT_EMPTY
    # other fits against the oracle on the decoded FP32 samples
    from types import SimpleNamespace
    b = SimpleNamespace(offsets=off, x=x32, y=y, n_vars=3, degree=2, n_scale_log2=23,
                        b_scale_log2=10)
    check(b, c8.cpu().numpy().astype(np.float64), st, "df32", 0)
    # a block-size scale outside the binned kernel's range: the per-sample
    # kernel reads the same bytes (both scalings are exact)
    kw11 = dict(kw, b_scale_log2=16)
    c8b, s8b, _ = ctx.fit(t(off), t(x8), t(y), **kw11)
    c32b, s32b, _ = ctx.fit(t(off), t(x32), t(y), **kw11)
    torch.cuda.synchronize()
    assert torch.equal(c8b, c32b) and torch.equal(s8b, s32b)
    # unsupported combinations are refused before anything runs
    for bad in (dict(kw, precision=klr.FIT_FP64), dict(kw, refine_iters=1), dict(kw, degree=3)):
        with pytest.raises(klr.KlrError) as e_:
            ctx.fit(t(off), t(x8), t(y), **bad)
        assert e_.value.status == klr.ENOTSUP


def test_exp16_samples_equal_float32_samples(klr, ctx):
    """KLR_EXP16 (one 16-bit code per sample: log2 N | log2 b0 << 6 | log2 b1
    << 11) carries the same power-of-two samples in 6 bytes: every output
    equals the FP32-input fit's bit for bit, the per-sample route included (a
    fit with an N outside the 16 binned octaves, N = 2^63 at the code's top,
    an empty fit, and a block-size scale outside the binned kernel's range)."""
    fb = W.fit_batch(30, 3, (50, 900), noise=0.01, dtype=np.float32)
    e = np.round(np.log2(fb.x.astype(np.float64))).astype(np.int64)
    assert np.array_equal(np.ldexp(1.0, e), fb.x)
    e[0, fb.offsets[2]] = 6                       # N = 64: per-sample route
    e[0, fb.offsets[6] + 3] = 63                  # N = 2^63, the largest code
    code = (e[0] | (e[1] << 6) | (e[2] << 11)).astype(np.uint16).view(np.int16)
    x32 = np.ldexp(1.0, e).astype(np.float32)
    off = fb.offsets.copy()
    off[9:] = off[9:] - (off[9] - off[8])         # fit 8 empty
    keep = np.r_[0:fb.offsets[8], fb.offsets[9]:fb.offsets[-1]]
    code, x32, y = code[keep], x32[:, keep], fb.y[keep]
    t = lambda a: torch.tensor(np.ascontiguousarray(a)).cuda()
    kw = dict(n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10, precision=klr.FIT_DF32,
              refine_iters=0, coef_dtype=klr.F32)
    c16, s16, d16 = ctx.fit(t(off), t(code), t(y), **kw)
    c32, s32, d32 = ctx.fit(t(off), t(x32), t(y), **kw)
    torch.cuda.synchronize()
    assert torch.equal(c16, c32) and torch.equal(s16, s32) and torch.equal(d16, d32)
    st = s16.cpu().numpy()
    assert st[8] == rational.FIT_EMPTY
    kw16 = dict(kw, b_scale_log2=16)
    c16b, s16b, _ = ctx.fit(t(off), t(code), t(y), **kw16)
    c32b, s32b, _ = ctx.fit(t(off), t(x32), t(y), **kw16)
    torch.cuda.synchronize()
    assert torch.equal(c16b, c32b) and torch.equal(s16b, s32b)
    for bad in (dict(kw, precision=klr.FIT_FP64), dict(kw, refine_iters=1), dict(kw, degree=3)):
        with pytest.raises(klr.KlrError) as e_:
            ctx.fit(t(off), t(code), t(y), **bad)
        assert e_.value.status == klr.ENOTSUP


def test_degree3_refinement(klr, ctx):
    fb = W.fit_batch(24, 2, 1500, degree=3, n_hi_log2=30, dtype=np.float64)
    ref = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 3, 30, 10)
    errs = []
    for refine in (0, 1, 2):
        coef, st, _ = gpu_fit(klr, ctx, fb, klr.FIT_FP64, refine)
        errs.append(check(fb, coef, st, "fp64", refine, ref))
    assert errs[2] <= errs[0]


@pytest.mark.parametrize("refine", [0, 1])
def test_3d_blocks_degree2(klr, ctx, refine):
    # refine 0 runs the lane-per-fit solver, refine 1 the warp solver + passes
    fb = W.fit_batch(25, 3, 400, n_vars=4, noise=0.01, dtype=np.float32)
    coef, st, _ = gpu_fit(klr, ctx, fb, klr.FIT_DF32, refine)
    check(fb, coef, st, "df32", refine)


def test_fp32_mode_runs_and_reports(klr, ctx):
    fb = W.fit_batch(26, 2, 500, noise=0.01, dtype=np.float32)
    coef, st, diag = gpu_fit(klr, ctx, fb, klr.FIT_FP32, 2)
    assert np.all(np.isfinite(coef))
    assert np.allclose(np.linalg.norm(coef, axis=1), 1.0, atol=1e-12)


def test_edge_cases(klr, ctx):
    # fit 0 empty, fit 1 has a NaN, fit 2 all samples at one point, fit 3 too few,
    # fit 4 a regular noiseless fit
    base = W.fit_batch(27, 1, 60, dtype=np.float64)
    xs, ys, offs = [], [], [0]
    xs.append(np.zeros((3, 0))); ys.append(np.zeros(0))
    x1 = base.x[:, :30].copy(); y1 = base.y[:30].copy(); y1[7] = np.nan
    xs.append(x1); ys.append(y1)
    xs.append(np.tile(np.array([[4096.0], [32.0], [4.0]]), (1, 50))); ys.append(np.full(50, 1.5))
    xs.append(base.x[:, :12]); ys.append(base.y[:12])
    xs.append(base.x[:, :60]); ys.append(base.y[:60])
    for a in ys:
        offs.append(offs[-1] + len(a))
    fb = W.FitBatch(3, 2, 23, 10, np.array(offs, dtype=np.int64), np.hstack(xs), np.hstack(ys),
                    base.truth)
    coef, st, _ = gpu_fit(klr, ctx, fb, klr.FIT_FP64, 0)
    assert st[0] == klr.FIT_EMPTY and np.all(coef[0] == 0)
    assert st[1] == klr.FIT_NONFINITE and np.all(coef[1] == 0)
    assert st[2] & klr.FIT_RANK_DEFICIENT
    assert st[3] & klr.FIT_RANK_DEFICIENT
    assert st[4] == 0
    oc, ost, _ = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, 23, 10)
    assert ost[0] == rational.FIT_EMPTY and ost[1] == rational.FIT_NONFINITE
    assert np.max(np.abs(coef[4] - oc[4])) < 1e-7
    # zero fits is a no-op
    z = W.FitBatch(3, 2, 23, 10, np.zeros(1, dtype=np.int64), np.zeros((3, 1)), np.zeros(1),
                   base.truth)
    c0, s0, _ = gpu_fit(klr, ctx, z, klr.FIT_FP64, 0)
    assert c0.shape == (0, 20)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tensor_core_gram_edge_cases(klr, ctx, mode):
    """The tcgen05 Gram's per-fit cases: an empty fit between others (its
    tensor memory is not read), a NaN sample, a fit of 1 sample, ragged counts
    (not multiples of the 64-sample tile) and one of 130 samples (three tiles
    over two buffers); the statuses equal the oracle's, and a degree-1 fit
    whose gap leaves room for the operand rounding meets the bound after
    refinement."""
    base = W.fit_batch(44, 1, 400, degree=1, dtype=np.float64)
    xs, ys = [], []
    xs.append(base.x[:, :130]); ys.append(base.y[:130])
    xs.append(np.zeros((3, 0))); ys.append(np.zeros(0))
    x2 = base.x[:, 130:190].copy(); y2 = base.y[130:190].copy(); y2[11] = np.nan
    xs.append(x2); ys.append(y2)
    xs.append(base.x[:, 190:191]); ys.append(base.y[190:191])
    xs.append(base.x[:, 191:400]); ys.append(base.y[191:400])
    offs = np.concatenate([[0], np.cumsum([len(a) for a in ys])]).astype(np.int64)
    fb = W.FitBatch(3, 1, 23, 10, offs, np.hstack(xs), np.hstack(ys), base.truth)
    prec = klr.FIT_TF32 if mode == "tf32" else klr.FIT_BF16
    coef, st, _ = gpu_fit(klr, ctx, fb, prec, 6)
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 1, 23, 10)
    assert st[1] == klr.FIT_EMPTY and np.all(coef[1] == 0)
    assert st[2] == klr.FIT_NONFINITE and np.all(coef[2] == 0)
    assert st[3] & klr.FIT_RANK_DEFICIENT
    assert ost[1] == rational.FIT_EMPTY and ost[2] == rational.FIT_NONFINITE
    eps = 2.0 ** -11 if mode == "tf32" else 2.0 ** -8
    for f in (0, 4):
        assert (st[f] & ~klr.FIT_RANK_DEFICIENT) == 0
        gap = od[f][1] ** 2 - od[f][0] ** 2
        if eps / gap < 0.02:
            assert np.max(np.abs(coef[f] - oc[f])) <= 1e-9


def test_bad_arguments(klr, ctx):
    fb = W.fit_batch(28, 1, 50, dtype=np.float64)
    with pytest.raises(klr.KlrError) as e:
        gpu_fit(klr, ctx, fb, klr.FIT_DF32, 0)        # DF32 needs FP32 samples
    assert e.value.status == klr.EINVAL
    with pytest.raises(klr.KlrError) as e:
        gpu_fit(klr, ctx, fb, klr.FIT_FP64, 9)
    assert e.value.status == klr.EINVAL


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_tensor_core_gram_with_refinement(klr, ctx, mode):
    # Gram products on tensor cores with TF32/BF16 operands, then FP64
    # refinement passes over the samples.  Each pass contracts the error by
    # about eps / gap (eps = 2^-11 for TF32, 2^-8 for BF16): on the fits where
    # that is small the passes reach the FP64 answer; elsewhere they cannot.
    fb = W.fit_batch(43, 8, 400, degree=1, n_lo_log2=8, n_hi_log2=23, dtype=np.float64)
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 1, 23, 10)
    gap = od[:, 1] ** 2 - od[:, 0] ** 2
    eps = 2.0 ** -11 if mode == "tf32" else 2.0 ** -8
    prec = klr.FIT_TF32 if mode == "tf32" else klr.FIT_BF16
    errs = {}
    for refine in (0, 2, 6):
        coef, st, diag = gpu_fit(klr, ctx, fb, prec, refine)
        assert np.all(st & ~klr.FIT_RANK_DEFICIENT == 0)
        assert np.allclose(np.linalg.norm(coef, axis=1), 1.0, atol=1e-12)
        assert np.all(diag[:, 3] == refine)
        errs[refine] = np.max(np.abs(coef - oc), axis=1)
    good = eps / gap < 0.02
    if mode == "tf32":
        assert good.sum() >= 4   # this seeded batch has six such fits
    if good.any():
        assert np.all(errs[6][good] <= 1e-9), errs[6][good]
        assert np.all(errs[6][good] <= errs[0][good] + 1e-12)


def test_fp64_refinement_in_small_and_large_batches(klr, ctx):
    """A batch of at most one fit per SM gives each fit a block (four warps
    in the FP64 moments and in the refinement passes); a larger one packs
    four fits per block, one warp each.  The same noisy fits solved both ways
    (20 kernels = 160 fits, then the first 8 alone) meet the derived bound
    64 u eps / gap, agree with each other within twice it, and one pass
    lowers the median error (by about 50x here).  A single fit's refined
    error can exceed its unrefined one: the pass converges to the fixed
    point of the FP64 residual over the samples, whose rounding is of the
    order of the bound (one fit of this batch goes from 1e-12 to 5e-11, in
    this build and in the one before the four-warp passes alike)."""
    fb = W.fit_batch(29, 20, (200, 600), noise=0.01, dtype=np.float64)
    assert len(fb.offsets) - 1 > torch.cuda.get_device_properties(0).multi_processor_count
    oc, ost, od = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, 23, 10)
    ref = (oc, ost, od)
    gap = np.maximum(od[:, 1] ** 2 - od[:, 0] ** 2, 1e-300)
    b0 = np.maximum(64.0 * 20 * EPS["fp64"] / gap, 1e-11)
    coef_0, st_0, _ = gpu_fit(klr, ctx, fb, klr.FIT_FP64, 0)
    coef_l, st_l, diag_l = gpu_fit(klr, ctx, fb, klr.FIT_FP64, 1)
    check(fb, coef_l, st_l, "fp64", 0, ref)
    assert np.all(diag_l[:, 3] == 1)
    e0 = np.max(np.abs(coef_0 - oc), axis=1)
    e1 = np.max(np.abs(coef_l - oc), axis=1)
    assert np.median(e1) <= 0.1 * np.median(e0)
    n = 8
    e = int(fb.offsets[n])
    small = W.FitBatch(fb.n_vars, fb.degree, fb.n_scale_log2, fb.b_scale_log2,
                       fb.offsets[:n + 1].copy(), np.ascontiguousarray(fb.x[:, :e]),
                       fb.y[:e].copy(), fb.truth)
    coef_s, st_s, _ = gpu_fit(klr, ctx, small, klr.FIT_FP64, 1)
    check(small, coef_s, st_s, "fp64", 0, (oc[:n], ost[:n], od[:n]))
    assert np.array_equal(st_s, st_l[:n])
    assert np.all(np.max(np.abs(coef_s - coef_l[:n]), axis=1) <= 2.0 * b0[:n])


def test_page_locked_host_inputs_give_the_same_fit(klr, ctx):
    """klr_fit's samples and offsets may be page-locked host memory, read in
    place by the kernels: the outputs equal those of the same inputs in
    device memory bit for bit; an ordinary host tensor is refused."""
    fb = W.fit_batch(31, 4, (50, 600), noise=0.01, dtype=np.float32)
    kw = dict(n_vars=3, degree=2, n_scale_log2=23, b_scale_log2=10, precision=klr.FIT_DF32,
              refine_iters=0, coef_dtype=klr.F32)
    h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    off_h, x_h, y_h = h(fb.offsets), h(fb.x), h(fb.y)
    c_h, s_h, d_h = ctx.fit(off_h, x_h, y_h, **kw)
    c_d, s_d, d_d = ctx.fit(off_h.cuda(), x_h.cuda(), y_h.cuda(), **kw)
    torch.cuda.synchronize()
    assert c_h.is_cuda and torch.equal(c_h, c_d) and torch.equal(s_h, s_d) and torch.equal(d_h, d_d)
    with pytest.raises(ValueError):
        ctx.fit(torch.from_numpy(fb.offsets), x_h, y_h, **kw)
