"""Oracle: the configuration set F (test infrastructure only).

Section IV defines F as the finite set of integer tuples a program parameter can
take; for CUDA the product of the block dimensions is a multiple of the warp size
(32) and at most the maximum threads per block (Section IV, step 1 remark and
step 4 remark (ii)); Section V adds that block dimensions are typically powers of
two.  F here is every tuple of powers of two whose product T satisfies
min_threads <= T <= max_threads and T % 32 == 0, ordered by T, then by
decreasing first dimension, then decreasing second.
"""
from __future__ import annotations

import itertools


def enumerate_configs(dims: int, min_threads: int = 32, max_threads: int = 1024):
    """List of block shapes (b0, b1[, b2]) as tuples of ints."""
    out = []
    max_e = max_threads.bit_length()
    for shape in itertools.product([1 << e for e in range(max_e)], repeat=dims):
        t = 1
        for b in shape:
            t *= b
        if min_threads <= t <= max_threads and t % 32 == 0:
            out.append(shape)
    out.sort(key=lambda s: (_prod(s), tuple(-b for b in s)))
    return out


def _prod(s):
    t = 1
    for b in s:
        t *= b
    return t
