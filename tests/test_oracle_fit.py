"""Pins of the oracle's rational fit (Section V-E; Section IV step 2).

* exact recovery of seeded ground-truth rational functions from noiseless
  samples (the closed form the paper states: exact values determine g);
* optimality invariants of the least-squares null vector on noisy data;
* equilibration, sign and rank-deficiency rules;
* degree 0 against its closed form.
"""
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
