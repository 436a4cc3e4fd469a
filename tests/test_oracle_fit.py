"""Pins of the oracle's rational fit (Section V-E; Section IV step 2).

* exact recovery of seeded ground-truth rational functions from noiseless
  samples (the closed form the paper states: exact values determine g);
* optimality invariants of the least-squares null vector on noisy data;
* equilibration, sign and rank-deficiency rules;
* degree 0 against its closed form;
* a mutation test: eleven plausible mistakes (a dropped sign, a wrong scale
  or exponent, transposed variables, the wrong singular vector, p and q
  swapped, ...) planted one at a time in a private copy of
  ``oracle.rational``, each of which must break at least one of these pins.
"""
import itertools
import math

import numpy as np
import pytest

import workloads as W
from oracle import rational

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _truth_normalised(coef, m):
    c = coef / np.linalg.norm(coef)
    return c * np.sign(c[m])


def test_basis_order_and_count():
    e = rational.monomial_exponents(3, 2)
    assert e == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0),
                 (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]
    for nv, d in [(3, 3), (4, 2), (4, 3), (2, 1)]:
        assert len(rational.monomial_exponents(nv, d)) == math.comb(nv + d, d)
    # the generator's independent term list uses the same documented order
    assert [tuple(t) for t in W.term_exponents(3, 3)] == rational.monomial_exponents(3, 3)


@pytest.mark.parametrize("degree,n_hi,count", [(2, 23, 200), (3, 30, 1200)])
def test_exact_recovery_noiseless(degree, n_hi, count):
    fb = W.fit_batch(7, 1, count, degree=degree, n_hi_log2=n_hi, dtype=np.float64)
    coef, status, diag = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, degree,
                                            fb.n_scale_log2, fb.b_scale_log2)
    m = rational.n_monomials(3, degree)
    exps = rational.monomial_exponents(3, degree)
    # evaluation grid: log-spaced sizes x every block shape
    sizes = W.log_spaced_sizes(64, 8, n_hi)
    shapes = np.ldexp(1.0, W.block_shape_exponents(2))
    pts = np.array([(n, b0, b1) for n in sizes for (b0, b1) in shapes], dtype=np.float64)
    xs = rational.scale_variables(pts, n_hi, 10)
    tol = 1e-9 if degree == 2 else 1e-7
    for f in range(fb.n_fits):
        assert status[f] == rational.FIT_OK
        truth = _truth_normalised(fb.truth.coef[0, f], m)
        assert np.max(np.abs(coef[f] - truth)) <= tol
        pr = rational.predict(coef[f], xs, exps)
        pt = rational.predict(truth, xs, exps)
        assert np.max(np.abs(pr - pt) / np.abs(pt).max()) <= 1e-10
        assert diag[f][0] < 1e-12 < diag[f][1]


def test_noisy_fit_is_least_squares_optimal():
    fb = W.fit_batch(9, 2, 300, noise=0.01, dtype=np.float64)
    coef, status, _ = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, 23, 10)
    m = 10
    exps = rational.monomial_exponents(3, 2)
    rng = np.random.default_rng(0)
    for f in range(fb.n_fits):
        a, b = fb.offsets[f], fb.offsets[f + 1]
        A = rational.design_matrix(rational.scale_variables(fb.x[:, a:b].T, 23, 10),
                                   fb.y[a:b], exps)
        d = rational.equilibration(A)
        v = coef[f] / d
        v /= np.linalg.norm(v)
        r0 = np.linalg.norm(A * d @ v)
        # the ground truth and random perturbations never do better
        t = fb.truth.coef[f // 8, f % 8] / d
        assert np.linalg.norm(A * d @ (t / np.linalg.norm(t))) >= r0
        for _ in range(50):
            w = v + 1e-3 * rng.standard_normal(2 * m)
            assert np.linalg.norm(A * d @ (w / np.linalg.norm(w))) >= r0 * (1 - 1e-12)
        # stationarity: v is an eigenvector of (AD)^T (AD)
        G = (A * d).T @ (A * d)
        lam = v @ G @ v
        assert np.linalg.norm(G @ v - lam * v) <= 1e-9 * np.linalg.norm(G)
        assert status[f] == rational.FIT_OK
        assert abs(np.linalg.norm(coef[f]) - 1) < 1e-14 and coef[f][m] > 0


def test_equilibration_power_of_two_and_range():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((50, 6)) * np.ldexp(1.0, rng.integers(-40, 40, 6))
    A[:, 2] = 0.5
    A[:, 3] = 0.0
    d = rational.equilibration(A)
    for j in range(6):
        m_, e = math.frexp(d[j])
        assert m_ == 0.5
        if j == 3:
            assert d[j] == 1.0
            continue
        sq = np.sum((A[:, j] * d[j]) ** 2)
        assert 0.5 <= sq < 2.0
    # column of fifty 0.5s: sum of squares 12.5 = 0.78 * 2^4 -> scale 2^-2
    assert d[2] == 0.25


def test_degree_zero_closed_form():
    # p = alpha, q = beta: A = [1 | -y]; for constant y the null vector is exact
    y = np.full(10, 0.375)
    x = np.ones((3, 10))
    c, st, _ = rational.fit_one(x, y, 3, 0, 0, 0)
    assert st == rational.FIT_OK
    assert c[0] / c[1] == pytest.approx(0.375, rel=1e-15)
    # for varying y the fit is the smallest eigenvector of the 2x2 equilibrated Gram
    y = np.array([1.0, 2.0, 3.0, 5.0])
    c, st, _ = rational.fit_one(np.ones((3, 4)), y, 3, 0, 0, 0)
    A = np.stack([np.ones(4), -y], 1)
    # squared norms 4 = 0.5*2^3 -> 2^-1, 39 = 0.61*2^6 -> 2^-3
    d = np.array([0.5, 0.125])
    G = (A * d).T @ (A * d)
    # closed form of the smallest eigenvector of a symmetric 2x2 matrix
    a, b, cc = G[0, 0], G[0, 1], G[1, 1]
    lam = 0.5 * (a + cc) - math.sqrt(0.25 * (a - cc) ** 2 + b * b)
    v = np.array([b, lam - a])
    want = d * v
    want /= np.linalg.norm(want)
    want *= np.sign(want[1])
    assert np.allclose(c, want, rtol=1e-13, atol=1e-15)


def test_status_flags():
    x = np.ones((3, 0))
    assert rational.fit_one(x, np.zeros(0), 3, 2, 23, 10)[1] == rational.FIT_EMPTY
    x = np.full((3, 5), 64.0)
    y = np.array([1.0, 2.0, np.nan, 1.0, 1.0])
    assert rational.fit_one(x, y, 3, 2, 23, 10)[1] == rational.FIT_NONFINITE
    # every sample at one point: a null space of dimension u - 1
    x = np.tile(np.array([[1024.0], [32.0], [2.0]]), (1, 40))
    y = np.full(40, 3.0)
    assert rational.fit_one(x, y, 3, 2, 23, 10)[1] & rational.FIT_RANK_DEFICIENT
    # fewer samples than unknowns - 1
    fb = W.fit_batch(3, 1, 12, dtype=np.float64)
    _, st, _ = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, 23, 10, fits=[0])
    assert st[0] & rational.FIT_RANK_DEFICIENT


def test_sign_rule_and_sample_permutation():
    fb = W.fit_batch(11, 1, 150, noise=0.02, dtype=np.float64)
    a, b = fb.offsets[0], fb.offsets[1]
    c1, _, _ = rational.fit_one(fb.x[:, a:b], fb.y[a:b], 3, 2, 23, 10)
    perm = np.random.default_rng(0).permutation(b - a)
    c2, _, _ = rational.fit_one(fb.x[:, a:b][:, perm], fb.y[a:b][perm], 3, 2, 23, 10)
    assert np.allclose(c1, c2, rtol=0, atol=1e-12)
    # scaling y by 2 doubles the fitted function
    c3, _, _ = rational.fit_one(fb.x[:, a:b], 2 * fb.y[a:b], 3, 2, 23, 10)
    exps = rational.monomial_exponents(3, 2)
    xs = rational.scale_variables(fb.x[:, a:b].T, 23, 10)
    assert np.allclose(rational.predict(c3, xs, exps), 2 * rational.predict(c1, xs, exps),
                       rtol=1e-9)


def test_box_basis_is_the_per_variable_bounds():
    from oracle import rational
    for n_vars, vd in ((3, (1, 1, 1)), (3, (2, 1, 1)), (3, (3, 1, 0)), (4, (2, 1, 1, 1))):
        exps = rational.monomial_exponents(n_vars, 0, vd)
        want = set(itertools.product(*[range(d + 1) for d in vd]))
        assert set(exps) == want and len(exps) == len(want)
        keys = [(sum(e), tuple(-v for v in e)) for e in exps]
        assert keys == sorted(keys)                 # graded, then decreasing tuples
        assert exps[0] == (0,) * n_vars
    # the box (d, d, d) contains the total-degree-d basis
    assert set(rational.monomial_exponents(3, 2)) <= set(rational.monomial_exponents(3, 0, (2, 2, 2)))


def test_box_basis_exact_recovery():
    from oracle import rational
    vd = (2, 1, 1)
    fb = W.fit_batch(51, 2, 150, degree=2, var_degree=vd, dtype=np.float64)
    coef, st, _ = rational.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, 23, 10, var_degree=vd)
    m = len(rational.monomial_exponents(3, 0, vd))
    assert coef.shape == (16, 2 * m) and np.all(st == 0)
    truth = fb.truth.coef.reshape(16, 2 * m)
    truth = truth / np.linalg.norm(truth, axis=1, keepdims=True)
    truth *= np.sign(truth[:, m:m + 1])
    assert np.max(np.abs(coef - truth)) < 1e-9


def test_relative_rms_closed_form_and_selection():
    from oracle import rational
    # p/q = (1 + x_N) / 2 on the constant-plus-N basis of the box (1, 0, 0)
    vd = (1, 0, 0)
    exps = rational.monomial_exponents(3, 0, vd)
    assert exps == [(0, 0, 0), (1, 0, 0)]
    coef = np.array([1.0, 1.0, 2.0, 0.0])
    N = np.array([2.0 ** 20, 2.0 ** 22, 2.0 ** 23])
    x = np.vstack([N, np.full(3, 32.0), np.full(3, 8.0)])
    g = (1 + N / 2.0 ** 23) / 2
    y = g * np.array([1.0, 1.1, 0.9])
    want = math.sqrt(np.mean(((g - y) / y) ** 2))
    assert abs(rational.relative_rms(coef, x, y, 3, 0, 23, 10, vd) - want) < 1e-15
    assert rational.relative_rms(coef, x, g, 3, 0, 23, 10, vd) == 0.0
    # held-out selection: the true box fits the held-out samples better than a
    # smaller box, and as well as a larger one
    fb = W.fit_batch(52, 1, 400, degree=2, var_degree=(2, 1, 1), dtype=np.float64)
    f = 3
    a, b = int(fb.offsets[f]), int(fb.offsets[f + 1])
    tr, ho = slice(a, a + 300), slice(a + 300, b)
    errs = {}
    for cand in ((1, 1, 1), (2, 1, 1), (3, 1, 1)):
        c, _, _ = rational.fit_one(fb.x[:, tr], fb.y[tr], 3, 0, 23, 10, cand)
        errs[cand] = rational.relative_rms(c, fb.x[:, ho], fb.y[ho], 3, 0, 23, 10, cand)
    assert errs[(2, 1, 1)] < 1e-9 and errs[(3, 1, 1)] < 1e-9 and errs[(1, 1, 1)] > 1e-4


def test_choose_basis_rule():
    from oracle import rational
    sizes = [8, 12, 16]
    E = np.array([[1e-3, 2e-12, 1e-12],      # both larger bases exact: the smaller of them
                  [9.3e-4, 9.4e-4, 9e-4],    # within 5% + floor of the least: the smallest
                  [1e-3, 5e-4, 4e-4],        # 5e-4 > 4.2e-4: only the largest qualifies
                  [np.nan, np.inf, 3e-3],    # non-finite never qualifies
                  [np.nan, np.nan, np.nan]])
    assert list(rational.choose_basis(E, sizes)) == [1, 0, 2, 2, -1]
    # equal sizes: the earlier candidate
    assert list(rational.choose_basis([[1e-6, 1e-6]], [8, 8])) == [0]


# ---------------------------------------------------------------------------
# The pins above, run against a private copy of ``oracle.rational`` in which
# one plausible mistake is planted at a time (on the CPU; the oracle itself is
# untouched): each mistake must break at least one pin.

def _pin_failures(mod):
    """Names of the pins that ``mod`` (a copy of oracle.rational) fails."""
    failed = []

    def pin(name, fn):
        try:
            if not fn():
                failed.append(name)
        except Exception:  # a crash is a failure of the pin
            failed.append(name)

    def basis_order():
        return mod.monomial_exponents(3, 2) == [
            (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0),
            (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]

    def exact_recovery():
        fb = W.fit_batch(7, 1, 200, degree=2, dtype=np.float64)
        coef, status, _ = mod.fit_batch(fb.offsets, fb.x, fb.y, 3, 2, fb.n_scale_log2,
                                        fb.b_scale_log2)
        for f in range(fb.n_fits):
            truth = _truth_normalised(fb.truth.coef[0, f], 10)
            if status[f] != mod.FIT_OK or np.max(np.abs(coef[f] - truth)) > 1e-9:
                return False
        return True

    def equilibration():
        rng = np.random.default_rng(4)
        A = rng.standard_normal((50, 6)) * np.ldexp(1.0, rng.integers(-40, 40, 6))
        A[:, 2] = 0.5
        d = mod.equilibration(A)
        sq = np.sum((A * d) ** 2, axis=0)
        return d[2] == 0.25 and bool(np.all((sq >= 0.5) & (sq < 2.0)))

    def noisy_sign_norm_and_scaling():
        fb = W.fit_batch(11, 1, 150, noise=0.02, dtype=np.float64)
        a, b = fb.offsets[0], fb.offsets[1]
        c1, _, _ = mod.fit_one(fb.x[:, a:b], fb.y[a:b], 3, 2, 23, 10)
        c3, _, _ = mod.fit_one(fb.x[:, a:b], 2 * fb.y[a:b], 3, 2, 23, 10)
        exps = mod.monomial_exponents(3, 2)
        xs = mod.scale_variables(fb.x[:, a:b].T, 23, 10)
        return (abs(np.linalg.norm(c1) - 1) < 1e-14 and c1[10] > 0
                and np.allclose(mod.predict(c3, xs, exps), 2 * mod.predict(c1, xs, exps),
                                rtol=1e-9))

    def degree_zero():
        c, st, _ = mod.fit_one(np.ones((3, 10)), np.full(10, 0.375), 3, 0, 0, 0)
        return st == mod.FIT_OK and abs(c[0] / c[1] - 0.375) <= 1e-15

    def status_flags():
        x = np.tile(np.array([[1024.0], [32.0], [2.0]]), (1, 40))
        return (mod.fit_one(np.ones((3, 0)), np.zeros(0), 3, 2, 23, 10)[1] == mod.FIT_EMPTY
                and bool(mod.fit_one(x, np.full(40, 3.0), 3, 2, 23, 10)[1]
                         & mod.FIT_RANK_DEFICIENT))

    for name, fn in [("basis order", basis_order), ("exact recovery", exact_recovery),
                     ("equilibration", equilibration),
                     ("sign, norm and scaling", noisy_sign_norm_and_scaling),
                     ("degree zero", degree_zero), ("status flags", status_flags)]:
        pin(name, fn)
    return failed


# (original text in oracle/rational.py, planted mistake)
FIT_MUTATIONS = [
    ("for e in itertools.product(range(d, -1, -1), repeat=n_vars):",
     "for e in itertools.product(range(d + 1), repeat=n_vars):"),
    ("xs[..., 0] = x[..., 0] * math.ldexp(1.0, -n_scale_log2)",
     "xs[..., 0] = x[..., 0] * math.ldexp(1.0, -b_scale_log2)"),
    ("for var, p in enumerate(e):", "for var, p in enumerate(reversed(e)):"),
    ("return np.hstack([phi, -np.asarray(y, dtype=np.float64)[:, None] * phi])",
     "return np.hstack([phi, np.asarray(y, dtype=np.float64)[:, None] * phi])"),
    ("d[j] = math.ldexp(1.0, -(e // 2))", "d[j] = math.ldexp(1.0, -e)"),
    ("c = c / np.linalg.norm(c)", "c = c / np.abs(c).max()"),
    ("s = 1.0 if q[0] > 0 else -1.0", "s = 1.0 if q[0] < 0 else -1.0"),
    ("c = normalise(d * vt[-1], m)", "c = normalise(vt[-1], m)"),
    ("c = normalise(d * vt[-1], m)", "c = normalise(d * vt[-2], m)"),
    ("if sfull[u - 2] <= RANK_TOL * sfull[0]:", "if sfull[u - 1] <= RANK_TOL * sfull[0]:"),
    ("return np.sum(phi * coef[..., :m], axis=-1) / np.sum(phi * coef[..., m:], axis=-1)",
     "return np.sum(phi * coef[..., m:], axis=-1) / np.sum(phi * coef[..., :m], axis=-1)"),
]


def _planted(orig, planted):
    import os
    import types
    path = os.path.join(os.path.dirname(rational.__file__), "rational.py")
    src = open(path).read()
    assert src.count(orig) == 1, f"oracle/rational.py no longer holds {orig!r} once"
    mod = types.ModuleType("oracle._planted_rational")
    mod.__package__ = "oracle"
    exec(compile(src.replace(orig, planted), path + " (planted)", "exec"), mod.__dict__)
    return mod


def test_fit_pins_pass_on_the_oracle():
    assert _pin_failures(rational) == []


@pytest.mark.parametrize("orig,planted", FIT_MUTATIONS)
def test_fit_pins_catch_planted_mistakes(orig, planted):
    assert _pin_failures(_planted(orig, planted)), f"no pin notices {planted!r}"
