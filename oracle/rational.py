"""Oracle: fitting a low-level metric as a rational function (test infrastructure only).

Section V-E: a metric is modelled as f = p/q, p and q polynomials in the
variables X_1..X_n with coefficients alpha (numerator) and beta (denominator).
Clearing the denominator at every sample (X_s, y_s) gives the homogeneous linear
system  p(X_s) - y_s q(X_s) = 0,  i.e.  [M_p | -y M_q] c = 0  with c = (alpha,
beta).  The matrix is a Vandermonde-like monomial matrix, ill-conditioned and
possibly rank-deficient, so the paper solves the least-squares problem by
singular value decomposition rather than QR.  Section IV, step 2 adds that with
exact values the function is recovered exactly (rational interpolation).

Readings of this project (the paper gives per-variable degree bounds and no
normalisation):
* the monomial basis is every monomial of total degree <= d in the scaled
  variables x = (N 2^-eN, b0 2^-eb, b1 2^-eb[, b2 2^-eb]), ordered by degree and
  then by decreasing exponent tuple (graded lexicographic);
* the homogeneous least-squares solution is the right singular vector of the
  column-equilibrated matrix A D for its smallest singular value, where D scales
  column j by the power of two 2^-floor(e_j / 2), e_j the binary exponent
  (frexp: sum_s A_sj^2 = f 2^e_j, f in [0.5, 1)) of the squared column norm, so
  the scaled squared norms lie in [0.5, 2) and the scaling is exact in binary;
  c = D v, normalised to unit 2-norm;
* sign: the denominator's constant coefficient is positive; if it is below
  1e-12 in magnitude, the largest-magnitude denominator coefficient (first on
  ties) is positive;
* the fit is flagged rank-deficient when the second-smallest singular value is
  at most 1e-12 of the largest (a null space of dimension > 1).

All arithmetic is float64; numpy.linalg.svd (LAPACK) is the SVD step.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

FIT_OK = 0
FIT_EMPTY = 1
FIT_NONFINITE = 2
FIT_RANK_DEFICIENT = 4

RANK_TOL = 1e-12
SIGN_TOL = 1e-12


def monomial_exponents(n_vars: int, degree: int, var_degree=None) -> list:
    """Exponent tuples of the basis, graded lex: every monomial of total degree
    <= degree, or, with per-variable bounds var_degree (Section V-E: the
    degree of each variable bounded separately), every monomial whose exponent
    of variable v is <= var_degree[v]."""
    if var_degree is not None and var_degree[0] > 0:
        bounds = [int(var_degree[v]) for v in range(n_vars)]
        out = [e for e in itertools.product(*[range(b, -1, -1) for b in bounds])]
        # by total degree, then decreasing exponent tuple
        return sorted((tuple(e) for e in out), key=lambda e: (sum(e), [-v for v in e]))
    out = []
    for d in range(degree + 1):
        for e in itertools.product(range(d, -1, -1), repeat=n_vars):
            if sum(e) == d:
                out.append(tuple(e))
    return out


def n_monomials(n_vars: int, degree: int) -> int:
    return math.comb(n_vars + degree, degree)


def scale_variables(x: np.ndarray, n_scale_log2: int, b_scale_log2: int) -> np.ndarray:
    """Raw rows (N, b0, b1[, b2]) -> scaled rows (power-of-two scaling)."""
    x = np.asarray(x, dtype=np.float64)
    xs = x * math.ldexp(1.0, -b_scale_log2)
    xs[..., 0] = x[..., 0] * math.ldexp(1.0, -n_scale_log2)
    return xs


def monomials(xs: np.ndarray, exps: list) -> np.ndarray:
    """(..., n_vars) scaled points -> (..., m) monomial values."""
    xs = np.asarray(xs, dtype=np.float64)
    out = np.empty(xs.shape[:-1] + (len(exps),))
    for t, e in enumerate(exps):
        v = np.ones(xs.shape[:-1])
        for var, p in enumerate(e):
            for _ in range(p):
                v = v * xs[..., var]
        out[..., t] = v
    return out


def design_matrix(xs: np.ndarray, y: np.ndarray, exps: list) -> np.ndarray:
    """A = [Phi | -y Phi], one row per sample."""
    phi = monomials(xs, exps)
    return np.hstack([phi, -np.asarray(y, dtype=np.float64)[:, None] * phi])


def equilibration(A: np.ndarray) -> np.ndarray:
    """Power-of-two column scales d_j = 2^-floor(e_j / 2), e_j = frexp exponent
    of sum_s A_sj^2 (1 for an all-zero column)."""
    d = np.ones(A.shape[1])
    for j in range(A.shape[1]):
        sq = float(np.sum(A[:, j] * A[:, j]))
        if sq > 0:
            _, e = math.frexp(sq)
            d[j] = math.ldexp(1.0, -(e // 2))
    return d


def normalise(c: np.ndarray, m: int) -> np.ndarray:
    """Unit 2-norm and the sign rule on the denominator."""
    c = c / np.linalg.norm(c)
    q = c[m:]
    if abs(q[0]) >= SIGN_TOL:
        s = 1.0 if q[0] > 0 else -1.0
    else:
        j = int(np.argmax(np.abs(q)))
        s = 1.0 if q[j] > 0 else -1.0
    return c * s


def fit_one(x: np.ndarray, y: np.ndarray, n_vars: int, degree: int,
            n_scale_log2: int, b_scale_log2: int, var_degree=None):
    """Fit one rational function.

    x: (n_vars, S) raw sample coordinates, y: (S,) metric values.
    Returns (coef (2m,), status, diag) with diag = (sigma_min/sigma_max,
    sigma_2nd_min/sigma_max, rms of A c over samples).
    """
    exps = monomial_exponents(n_vars, degree, var_degree)
    m = len(exps)
    u = 2 * m
    y = np.asarray(y, dtype=np.float64)
    S = y.shape[0]
    if S == 0:
        return np.zeros(u), FIT_EMPTY, np.zeros(3)
    xr = np.asarray(x, dtype=np.float64).T
    if not (np.all(np.isfinite(xr)) and np.all(np.isfinite(y))):
        return np.zeros(u), FIT_NONFINITE, np.zeros(3)
    A = design_matrix(scale_variables(xr, n_scale_log2, b_scale_log2), y, exps)
    d = equilibration(A)
    # right singular vectors of A D (U is not needed; with fewer samples than
    # unknowns the full V supplies the null space)
    _, s, vt = np.linalg.svd(A * d, full_matrices=S < u)
    sfull = np.zeros(u)
    sfull[:len(s)] = s
    c = normalise(d * vt[-1], m)
    status = FIT_OK
    if sfull[u - 2] <= RANK_TOL * sfull[0]:
        status |= FIT_RANK_DEFICIENT
    diag = np.array([sfull[u - 1] / sfull[0], sfull[u - 2] / sfull[0],
                     np.linalg.norm(A @ c) / math.sqrt(S)])
    return c, status, diag


def fit_batch(offsets, x, y, n_vars, degree, n_scale_log2, b_scale_log2, fits=None,
              var_degree=None):
    """Fit every fit f (or the subset ``fits``) of a CSR batch.

    offsets: (F+1,), x: (n_vars, S), y: (S,).  Returns coef (len, 2m), status,
    diag (len, 3)."""
    fits = range(len(offsets) - 1) if fits is None else fits
    m = len(monomial_exponents(n_vars, degree, var_degree))
    coef = np.zeros((len(fits), 2 * m))
    status = np.zeros(len(fits), dtype=np.int32)
    diag = np.zeros((len(fits), 3))
    for i, f in enumerate(fits):
        a, b = int(offsets[f]), int(offsets[f + 1])
        coef[i], status[i], diag[i] = fit_one(x[:, a:b], y[a:b], n_vars, degree,
                                              n_scale_log2, b_scale_log2, var_degree)
    return coef, status, diag


def predict(coef: np.ndarray, xs: np.ndarray, exps: list) -> np.ndarray:
    """p(x)/q(x) for coefficient rows (..., 2m) at scaled points (..., n_vars)."""
    m = len(exps)
    phi = monomials(xs, exps)
    return np.sum(phi * coef[..., :m], axis=-1) / np.sum(phi * coef[..., m:], axis=-1)


def relative_rms(coef: np.ndarray, x: np.ndarray, y: np.ndarray, n_vars: int, degree: int,
                 n_scale_log2: int, b_scale_log2: int, var_degree=None) -> float:
    """Root mean square of (p/q - y) / y over samples (x (n_vars, S) raw, y (S,)):
    the held-out error by which a basis is chosen."""
    exps = monomial_exponents(n_vars, degree, var_degree)
    xs = scale_variables(np.asarray(x, dtype=np.float64).T, n_scale_log2, b_scale_log2)
    y = np.asarray(y, dtype=np.float64)
    if y.size == 0:
        return 0.0
    g = predict(np.asarray(coef, dtype=np.float64), xs, exps)
    return float(np.sqrt(np.mean(((g - y) / y) ** 2)))



def choose_basis(errors: np.ndarray, sizes, tol: float = 0.05, floor: float = 1e-6) -> np.ndarray:
    """Per fit (row of errors, one column per candidate basis): the candidate
    with the fewest monomials (sizes; ties by column order) among those whose
    held-out error is <= (1 + tol) x the least error + floor.  A reading of
    Section V-E, which leaves the choice of degree bounds open: prefer the
    smaller model unless a larger one predicts held-out samples clearly
    better; errors below the floor (default 1e-6, above the relative rounding
    of FP32 samples) count as equal.  Non-finite errors never qualify (-1
    when none is finite)."""
    errors = np.atleast_2d(np.asarray(errors, dtype=np.float64))
    out = np.full(errors.shape[0], -1, dtype=np.int64)
    for f in range(errors.shape[0]):
        e = errors[f]
        fin = np.isfinite(e)
        if not fin.any():
            continue
        lim = e[fin].min() * (1.0 + tol) + floor
        ok = [j for j in range(len(e)) if fin[j] and e[j] <= lim]
        out[f] = min(ok, key=lambda j: (sizes[j], j))
    return out
