"""Pins of the seeded input generator shared by the oracle and the CUDA path.

* the stream words are SplitMix64 (Vigna's reference generator): a stream with
  key k yields the sequence the reference implementation yields from state k,
  checked against its published first outputs from state 0;
* uniform doubles fill [0, 1) with the moments of the uniform distribution,
  normals those of the standard normal (statistical bounds several standard
  errors wide, on a fixed seed, so the test is deterministic);
* the sampling domain of block shapes and the seeded batches are deterministic,
  inside the domain and independent of each other across seeds.
"""
import math

import numpy as np

import workloads as W


def test_words_are_splitmix64():
    # first three outputs of SplitMix64 from state 0
    got = W.words(np.uint64(0), np.arange(3, dtype=np.uint64))
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                     0x06C45D188009454F]
    # a stream key is the state: counters continue the same sequence
    k = np.uint64(W.stream_key(5, 1, 2))
    seq = W.words(k, np.arange(6, dtype=np.uint64))
    assert np.array_equal(W.words(k, np.arange(3, 6, dtype=np.uint64)), seq[3:])
    assert len(set(int(v) for v in seq)) == 6
    # the scalar and vectorised finalisers agree
    z = np.array([0, 1, 2 ** 63, 2 ** 64 - 1], dtype=np.uint64)
    assert [int(v) for v in W._mix(z)] == [W._mix_scalar(int(v)) for v in z]


def test_uniform_and_normal_moments():
    n = 400_000
    keys = np.uint64(W.stream_key(2024, 9))
    u = W.uniform(keys, np.arange(n, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    # standard errors: mean 1/sqrt(12 n), variance about 0.0745/sqrt(n)
    assert abs(u.mean() - 0.5) < 6 / math.sqrt(12 * n)
    assert abs(u.var() - 1 / 12) < 6 * 0.0745 / math.sqrt(n)
    # top 53 bits: every value is a multiple of 2^-53
    assert np.all(np.ldexp(u, 53) == np.floor(np.ldexp(u, 53)))
    g = W.normal(keys, np.arange(n, dtype=np.uint64))
    assert abs(g.mean()) < 6 / math.sqrt(n)
    assert abs(g.var() - 1.0) < 6 * math.sqrt(2.0 / n)
    # fourth moment 3 (standard error about sqrt(96 / n))
    assert abs(np.mean(g ** 4) - 3.0) < 6 * math.sqrt(96.0 / n)
    assert abs(np.mean(np.abs(g) < 1.0) - 0.6826894921370859) < 6 * math.sqrt(0.22 / n)


def test_block_shape_domain():
    e2 = W.block_shape_exponents(2)
    e3 = W.block_shape_exponents(3)
    assert len(e2) == 51 and len(e3) == 251
    for e in (e2, e3):
        s = e.sum(1)
        assert np.all((s >= 5) & (s <= 10)) and np.all(np.diff(s) >= 0)
        assert len({tuple(r) for r in e}) == len(e)


def test_fit_batches_are_seeded_and_in_domain():
    a = W.fit_batch(31, 3, (50, 120), noise=0.01, dtype=np.float32)
    b = W.fit_batch(31, 3, (50, 120), noise=0.01, dtype=np.float32)
    c = W.fit_batch(32, 3, (50, 120), noise=0.01, dtype=np.float32)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.x, b.x)
    assert np.array_equal(a.y, b.y)
    assert not np.array_equal(a.y[:50], c.y[:50])
    assert a.n_fits == 24 and np.all(np.diff(a.offsets) >= 50) and np.all(np.diff(a.offsets) <= 120)
    # N a power of two in [2^8, 2^23]; each block shape one of the 51
    n = a.x[0].astype(np.float64)
    assert np.all(np.exp2(np.round(np.log2(n))) == n) and n.min() >= 2 ** 8 and n.max() <= 2 ** 23
    shapes = {(1 << int(i), 1 << int(j)) for i, j in W.block_shape_exponents(2)}
    assert {(int(p), int(q)) for p, q in zip(a.x[1], a.x[2])} <= shapes
