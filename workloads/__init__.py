"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures its method on PolyBench/GPU kernels profiled on a GTX 1080Ti
(Section VI).  That suite and those profiles are not available here, so every
input of this project is synthetic, drawn from a counter-based generator, and
has the structure the paper describes:

* data sizes N are powers of two for the fit samples (Section V: "the values of
  which are usually powers of 2") and log-spaced integers for queries;
* thread-block shapes are powers of two whose product is a multiple of 32 and at
  most 1024 (Section IV, step 4, remark (ii); Section V);
* each low-level metric is a rational function p/q of (N, b) of bounded total
  degree (Section V-E), so noiseless samples determine it exactly (Section IV,
  step 2).

This module is the only code shared by the CUDA path's tests/bench and the
oracle.  It holds no arithmetic of the method itself: it draws numbers,
evaluates the seeded ground-truth functions that stand in for profiled metric
values, and lays the results out in the arrays the library consumes.

Generator: splitmix64 (S. Vigna's published finaliser) in counter mode.  A
stream key is derived from (seed, *ids) and the i-th 64-bit word of a stream is
``mix(key + (i + 1) * GAMMA)``.  Uniform doubles take the top 53 bits; normals
use the Box-Muller transform.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB
_MASK = (1 << 64) - 1

# Purpose ids for the generator's streams.
_S_COEF, _S_SAMPLES, _S_NOISE, _S_COUNTS, _S_RES, _S_MISC = 11, 12, 13, 14, 15, 16


def _mix_scalar(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * _M1) & _MASK
    z = ((z ^ (z >> 27)) * _M2) & _MASK
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(_M1)
        z ^= z >> np.uint64(27)
        z *= np.uint64(_M2)
        z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, *ids: int) -> int:
    """Key of the stream named by (seed, *ids)."""
    k = _mix_scalar(seed + GAMMA)
    for i in ids:
        k = _mix_scalar(k ^ ((int(i) + GAMMA) & _MASK))
    return k


def stream_keys(seed: int, ids_prefix: tuple, last: np.ndarray) -> np.ndarray:
    """Vectorised ``stream_key(seed, *ids_prefix, last[i])``."""
    k = stream_key(seed, *ids_prefix)
    last = np.asarray(last, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(k) ^ (last + np.uint64(GAMMA)))


def words(keys, counters) -> np.ndarray:
    """64-bit words ``mix(key + (counter + 1) * GAMMA)`` (broadcasting)."""
    keys = np.asarray(keys, dtype=np.uint64)
    counters = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(keys + (counters + np.uint64(1)) * np.uint64(GAMMA))


def uniform(keys, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each word."""
    w = words(keys, counters)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(keys, counters) -> np.ndarray:
    """Standard normals by Box-Muller from words 2c and 2c+1 of each stream."""
    counters = np.asarray(counters, dtype=np.uint64)
    u1 = uniform(keys, counters * np.uint64(2))
    u2 = uniform(keys, counters * np.uint64(2) + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# The input domain: block shapes and data sizes.
# ---------------------------------------------------------------------------

def block_shape_exponents(dims: int, min_log2: int = 5, max_log2: int = 10) -> np.ndarray:
    """Exponent tuples (i, j[, k]) of block shapes (2^i, 2^j[, 2^k]) whose thread
    count 2^(i+j[+k]) lies in [2^min_log2, 2^max_log2], listed by thread count,
    then by decreasing i, then decreasing j.  This is the sampling domain of the
    synthetic profiles; the library enumerates its own configuration table."""
    out = []
    for s in range(min_log2, max_log2 + 1):
        for e in itertools.product(range(s, -1, -1), repeat=dims):
            if sum(e) == s:
                out.append(e)
    return np.array(out, dtype=np.int64)


def log_spaced_sizes(count: int, lo_log2: int = 8, hi_log2: int = 23) -> np.ndarray:
    """``round(2^(lo + (hi-lo) * j / (count-1)))`` for j = 0..count-1 (rounded
    half away from zero)."""
    if count == 1:
        return np.array([1 << lo_log2], dtype=np.int64)
    j = np.arange(count, dtype=np.float64)
    v = np.exp2(lo_log2 + (hi_log2 - lo_log2) * j / (count - 1))
    return np.floor(v + 0.5).astype(np.int64)


def term_exponents(n_vars: int, degree: int, var_degree=None) -> np.ndarray:
    """Exponents of the ground-truth polynomial terms: total degree <= degree
    (or, with var_degree, exponent <= var_degree[v] in variable v), by total
    degree, then decreasing lexicographic order (the coefficient order the
    library documents)."""
    box = var_degree is not None and var_degree[0] > 0
    top = sum(int(v) for v in var_degree[:n_vars]) if box else degree
    out = []
    for d in range(top + 1):
        for e in itertools.product(range(d, -1, -1), repeat=n_vars):
            if sum(e) != d:
                continue
            if box and any(e[v] > var_degree[v] for v in range(n_vars)):
                continue
            out.append(e)
    return np.array(out, dtype=np.int64)


# ---------------------------------------------------------------------------
# Hardware vector and metric map (inputs of the rational program).
# ---------------------------------------------------------------------------

#: Hardware of the single-kernel workload: 148 SMs, 64 warps/SM, 64 Ki
#: registers/SM, 228 KiB shared memory/SM, 600-cycle memory latency, 8 TB/s,
#: 1.9 GHz.  Blocks/SM (32), threads/block (1024) and the coalesced/uncoalesced
#: departure delays (4 and 10 cycles) are fixed model constants of this project.
HARDWARE = dict(
    n_sm=148, max_warps_per_sm=64, regs_per_sm=65536, smem_per_sm=233472,
    max_blocks_per_sm=32, max_threads_per_block=1024,
    mem_latency=600.0, mem_bandwidth=8.0e12, clock_hz=1.9e9,
    departure_delay_coal=4.0, departure_delay_uncoal=10.0,
)

#: The eight low-level metrics, in order, with the map L = lo + s*|g| that turns
#: a fitted rational function g into a valid count.
METRIC_NAMES = ("comp_insts", "coal_mem_insts", "uncoal_mem_insts", "synch_insts",
                "coal_per_mw", "uncoal_per_mw", "load_bytes_per_warp", "issue_cycles")
METRIC_LO = (1.0, 1.0, 0.0, 0.0, 1.0, 1.0, 32.0, 1.0)
METRIC_SCALE = (256.0, 32.0, 8.0, 4.0, 4.0, 31.0, 480.0, 8.0)
N_METRICS = 8

REGS_CHOICES = np.array([32, 64, 128], dtype=np.int32)
SMEM_CHOICES = np.array([0, 16384, 49152], dtype=np.int32)


# ---------------------------------------------------------------------------
# Ground-truth rational functions.
# ---------------------------------------------------------------------------

def _monomials(x: np.ndarray, exps: np.ndarray) -> np.ndarray:
    """x: (..., n_vars) -> (..., n_terms) products x^e."""
    out = np.ones(x.shape[:-1] + (len(exps),), dtype=np.float64)
    for t, e in enumerate(exps):
        for v, p in enumerate(e):
            if p:
                out[..., t] *= x[..., v] ** int(p)
    return out


def _q_min_over_sizes(beta: np.ndarray, exps: np.ndarray, xb: np.ndarray,
                      xlo: float, xhi: float) -> np.ndarray:
    """Minimum over x_N in [xlo, xhi] of q(x_N, b) for every block shape row of
    ``xb`` (scaled b exponents already applied).  beta: (F, m).  Returns (F,)."""
    deg = int(exps[:, 0].max()) if len(exps) else 0
    # univariate coefficients in x_N for each (function, block shape)
    bmono = np.ones((xb.shape[0], len(exps)), dtype=np.float64)
    for t, e in enumerate(exps):
        for v, p in enumerate(e[1:]):
            if p:
                bmono[:, t] *= xb[:, v] ** int(p)
    qmin = np.full(beta.shape[0], np.inf)
    for s in range(xb.shape[0]):
        cu = np.zeros((beta.shape[0], deg + 1))
        for t, e in enumerate(exps):
            cu[:, e[0]] += beta[:, t] * bmono[s, t]
        pts = [np.full(beta.shape[0], xlo), np.full(beta.shape[0], xhi)]
        if deg >= 2:
            # stationary points of the univariate polynomial in [xlo, xhi]
            if deg == 2:
                with np.errstate(divide="ignore", invalid="ignore"):
                    r = -cu[:, 1] / (2.0 * cu[:, 2])
                pts.append(np.where(np.isfinite(r), np.clip(r, xlo, xhi), xlo))
            else:
                a, b, c = 3.0 * cu[:, 3], 2.0 * cu[:, 2], cu[:, 1]
                disc = np.maximum(b * b - 4 * a * c, 0.0)
                with np.errstate(divide="ignore", invalid="ignore"):
                    r1 = (-b + np.sqrt(disc)) / (2 * a)
                    r2 = (-b - np.sqrt(disc)) / (2 * a)
                    rl = -c / b
                for r in (r1, r2, rl):
                    pts.append(np.where(np.isfinite(r), np.clip(r, xlo, xhi), xlo))
        for xp in pts:
            val = np.zeros(beta.shape[0])
            for d in range(deg, -1, -1):
                val = val * xp + cu[:, d]
            qmin = np.minimum(qmin, val)
    return qmin


@dataclass
class GroundTruth:
    """Seeded ground-truth metric functions of ``n_kernels`` synthetic kernels."""
    n_vars: int
    degree: int
    n_scale_log2: int
    b_scale_log2: int
    coef: np.ndarray          # (n_kernels, 8, 2m) float64: [alpha (p) | beta (q)]
    regs: np.ndarray          # (n_kernels,) int32, registers per thread
    smem: np.ndarray          # (n_kernels,) int32, shared memory bytes per block
    attempts: np.ndarray = field(default=None)  # redraws used per (kernel, metric)
    var_degree: tuple = None  # per-variable degree bounds of the basis, or None

    @property
    def n_terms(self) -> int:
        return self.coef.shape[-1] // 2

    def values(self, kernel: np.ndarray, metric: np.ndarray, x: np.ndarray) -> np.ndarray:
        """g(x) = p(x)/q(x) for rows (kernel[i], metric[i], x[i] unscaled)."""
        exps = term_exponents(self.n_vars, self.degree, self.var_degree)
        xs = scale_points(x, self.n_scale_log2, self.b_scale_log2)
        phi = _monomials(xs, exps)
        c = self.coef[kernel, metric]
        m = self.n_terms
        return np.sum(phi * c[:, :m], axis=1) / np.sum(phi * c[:, m:], axis=1)


def scale_points(x: np.ndarray, n_scale_log2: int, b_scale_log2: int) -> np.ndarray:
    """Unscaled (N, b0, b1[, b2]) rows -> (N 2^-eN, b 2^-eb ...), exact in binary."""
    x = np.asarray(x, dtype=np.float64)
    s = np.full(x.shape[-1], np.ldexp(1.0, -b_scale_log2))
    s[0] = np.ldexp(1.0, -n_scale_log2)
    return x * s


def ground_truth(seed: int, n_kernels: int, n_vars: int = 3, degree: int = 2,
                 n_lo_log2: int = 8, n_hi_log2: int = 23, b_scale_log2: int = 10,
                 q_floor: float = 0.5, max_attempts: int = 64, kernels=None,
                 var_degree=None) -> GroundTruth:
    """Coefficients U(-1,1), +3 on the denominator's constant term, redrawn
    (next attempt id) until min q >= q_floor over every block shape and every
    N in [2^n_lo_log2, 2^n_hi_log2].  ``kernels`` selects a subset of the
    n_kernels kernel ids (same values as in the full set).  ``var_degree``:
    draw in the per-variable-bounds basis instead of the total-degree one."""
    exps = term_exponents(n_vars, degree, var_degree)
    m = len(exps)
    shapes = block_shape_exponents(n_vars - 1)
    xb = np.ldexp(1.0, shapes - b_scale_log2)
    xlo, xhi = np.ldexp(1.0, n_lo_log2 - n_hi_log2), 1.0
    kid = np.arange(n_kernels) if kernels is None else np.asarray(kernels, dtype=np.int64)
    n_kernels = len(kid)
    total = n_kernels * N_METRICS
    ids = (kid[:, None] * N_METRICS + np.arange(N_METRICS)[None, :]).reshape(-1).astype(np.uint64)
    coef = np.empty((total, 2 * m))
    attempts = np.zeros(total, dtype=np.int32)
    todo = np.arange(total)
    for a in range(max_attempts):
        keys = stream_keys(seed, (_S_COEF, a), ids[todo])
        cnt = np.arange(2 * m, dtype=np.uint64)
        draw = 2.0 * uniform(keys[:, None], cnt[None, :]) - 1.0
        draw[:, m] += 3.0
        ok = _q_min_over_sizes(draw[:, m:], exps, xb, xlo, xhi) >= q_floor
        coef[todo[ok]] = draw[ok]
        attempts[todo[ok]] = a
        todo = todo[~ok]
        if todo.size == 0:
            break
    if todo.size:
        raise RuntimeError(f"{todo.size} ground-truth functions failed the q floor")
    rk = stream_keys(seed, (_S_RES,), kid.astype(np.uint64))
    regs = REGS_CHOICES[(words(rk, 0) % np.uint64(3)).astype(np.int64)]
    smem = SMEM_CHOICES[(words(rk, 1) % np.uint64(3)).astype(np.int64)]
    return GroundTruth(n_vars, degree, n_hi_log2, b_scale_log2,
                       coef.reshape(n_kernels, N_METRICS, 2 * m),
                       regs.astype(np.int32), smem.astype(np.int32),
                       attempts.reshape(n_kernels, N_METRICS),
                       None if var_degree is None else tuple(int(v) for v in var_degree))


# ---------------------------------------------------------------------------
# Fit batches: ragged sample sets (CSR) of profiled metric values.
# ---------------------------------------------------------------------------

@dataclass
class FitBatch:
    """Samples of ``n_fits`` fits, fit f = (kernel f // 8, metric f % 8)."""
    n_vars: int
    degree: int
    n_scale_log2: int
    b_scale_log2: int
    offsets: np.ndarray   # (n_fits+1,) int64
    x: np.ndarray         # (n_vars, S) unscaled N, b0, b1[, b2] in `dtype`
    y: np.ndarray         # (S,) in `dtype`
    truth: GroundTruth

    @property
    def n_fits(self) -> int:
        return len(self.offsets) - 1


def fit_batch(seed: int, n_kernels: int, counts, n_vars: int = 3, degree: int = 2,
              n_lo_log2: int = 8, n_hi_log2: int = 23, b_scale_log2: int = 10,
              noise: float = 0.0, dtype=np.float32, replace: bool | None = None,
              truth: GroundTruth | None = None, kernels=None, var_degree=None) -> FitBatch:
    """Samples for every (kernel, metric) of a seeded ground truth.

    ``counts``: an int (same count for every fit) or a (lo, hi) pair, meaning a
    per-fit count drawn uniformly from the integers lo..hi.  Sample points are
    drawn from the grid {N = 2^k, n_lo_log2 <= k <= n_hi_log2} x block shapes,
    without replacement when the grid is large enough (else with replacement).
    ``y = g(x) * (1 + noise * eps)``, eps standard normal, then cast to dtype.
    """
    if truth is None:
        truth = ground_truth(seed, n_kernels, n_vars, degree, n_lo_log2, n_hi_log2,
                             b_scale_log2, kernels=kernels, var_degree=var_degree)
    kid = np.arange(n_kernels) if kernels is None else np.asarray(kernels, dtype=np.int64)
    n_fits = len(kid) * N_METRICS
    # global fit ids: the streams of a fit do not depend on which others are drawn
    fid = (kid[:, None] * N_METRICS + np.arange(N_METRICS)[None, :]).reshape(-1).astype(np.uint64)
    if isinstance(counts, (tuple, list)):
        lo, hi = counts
        ck = stream_keys(seed, (_S_COUNTS,), fid)
        cnt = lo + (words(ck, 0) % np.uint64(hi - lo + 1)).astype(np.int64)
    else:
        cnt = np.full(n_fits, int(counts), dtype=np.int64)
    offsets = np.zeros(n_fits + 1, dtype=np.int64)
    np.cumsum(cnt, out=offsets[1:])
    S = int(offsets[-1])
    shapes = block_shape_exponents(n_vars - 1)
    n_sizes = n_hi_log2 - n_lo_log2 + 1
    grid = n_sizes * len(shapes)
    # sample index within its fit
    fit_of = np.repeat(np.arange(n_fits, dtype=np.int64), cnt)
    local = np.arange(S, dtype=np.int64) - offsets[:-1][fit_of]
    keys = stream_keys(seed, (_S_SAMPLES,), fid)
    use_replace = (cnt.max(initial=0) > grid) if replace is None else replace
    if use_replace:
        pt = (words(keys[fit_of], local.astype(np.uint64)) % np.uint64(grid)).astype(np.int64)
    else:
        # Without replacement: rank grid points by a per-fit random key.  Fits are
        # processed in chunks to bound memory.
        pt = np.empty(S, dtype=np.int64)
        chunk = max(1, (1 << 24) // grid)
        gidx = np.arange(grid, dtype=np.uint64)
        for f0 in range(0, n_fits, chunk):
            f1 = min(n_fits, f0 + chunk)
            r = words(keys[f0:f1, None], gidx[None, :])
            order = np.argsort(r, axis=1, kind="stable")
            for f in range(f0, f1):
                pt[offsets[f]:offsets[f + 1]] = order[f - f0, :cnt[f]]
    k = n_lo_log2 + pt // len(shapes)
    sh = shapes[pt % len(shapes)]
    x = np.empty((n_vars, S), dtype=np.float64)
    x[0] = np.ldexp(1.0, k)
    x[1:] = np.ldexp(1.0, sh.T)
    # g on the whole grid for every fit, then gathered per sample
    gk = np.repeat(np.arange(n_lo_log2, n_hi_log2 + 1), len(shapes))
    gx = np.empty((grid, n_vars))
    gx[:, 0] = np.ldexp(1.0, gk)
    gx[:, 1:] = np.ldexp(1.0, np.tile(shapes, (n_sizes, 1)))
    phi = _monomials(scale_points(gx, n_hi_log2, b_scale_log2),
                     term_exponents(n_vars, degree, truth.var_degree))
    m = phi.shape[1]
    cf = truth.coef.reshape(n_fits, 2 * m)
    y = np.empty(S)
    step = max(1, (1 << 25) // grid)
    for f0 in range(0, n_fits, step):
        f1 = min(n_fits, f0 + step)
        g = (cf[f0:f1, :m] @ phi.T) / (cf[f0:f1, m:] @ phi.T)
        s0, s1 = offsets[f0], offsets[f1]
        y[s0:s1] = g[fit_of[s0:s1] - f0, pt[s0:s1]]
    if noise:
        nk = stream_keys(seed, (_S_NOISE,), fid)
        y = y * (1.0 + noise * normal(nk[fit_of], local.astype(np.uint64)))
    return FitBatch(n_vars, degree, n_hi_log2, b_scale_log2, offsets,
                    x.astype(dtype), y.astype(dtype), truth)


# ---------------------------------------------------------------------------
# Queries and the five workloads.
# ---------------------------------------------------------------------------

@dataclass
class Queries:
    """Per-kernel lists of data sizes (CSR by kernel)."""
    offsets: np.ndarray  # (n_kernels+1,) int64
    sizes: np.ndarray    # (n_q,) int64


def queries_per_kernel(n_kernels: int, sizes: np.ndarray) -> Queries:
    sizes = np.asarray(sizes, dtype=np.int64)
    return Queries(np.arange(n_kernels + 1, dtype=np.int64) * len(sizes),
                   np.tile(sizes, n_kernels))


def subsample_kernels(seed: int, n_kernels: int, count: int) -> np.ndarray:
    """A seeded sorted subset of ``count`` kernel ids (for bounded CPU checks)."""
    k = stream_keys(seed, (_S_MISC,), np.arange(n_kernels, dtype=np.uint64))
    r = words(k, 0)
    return np.sort(np.argsort(r, kind="stable")[:count])


WORKLOADS = {
    # name: (kernels, counts, n_vars, degree, n_hi_log2, noise, dtype, queries/kernel)
    "single_fp64": dict(n_kernels=1, counts=200, n_vars=3, degree=2, n_hi_log2=23,
                        noise=0.0, dtype=np.float64, n_query_sizes=16,
                        query_sizes="pow2"),
    "batched_fp32": dict(n_kernels=10000, counts=(50, 2000), n_vars=3, degree=2,
                         n_hi_log2=23, noise=0.01, dtype=np.float32,
                         n_query_sizes=64, query_sizes="log"),
    "precision_split": dict(n_kernels=512, counts=5000, n_vars=3, degree=3,
                            n_hi_log2=30, noise=0.0, dtype=np.float64,
                            n_query_sizes=64, query_sizes="log"),
    "sweep_3d": dict(n_kernels=100000, counts=0, n_vars=4, degree=2, n_hi_log2=23,
                     noise=0.0, dtype=np.float32, n_query_sizes=256,
                     query_sizes="log"),
}


def query_sizes(kind: str, count: int, lo_log2: int = 8, hi_log2: int = 23) -> np.ndarray:
    if kind == "pow2":
        return np.ldexp(1.0, np.arange(lo_log2, hi_log2 + 1)).astype(np.int64)[:count]
    return log_spaced_sizes(count, lo_log2, hi_log2)
