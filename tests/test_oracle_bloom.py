"""Pins of the oracle's interest vectors (Section 7): no false negatives, the
false-positive rate of a Bloom filter, and the window of deltas."""

import math

import numpy as np

import oracle
from paper_2001_08250_gb300 import synth


def test_no_false_negatives():
    m, k = 1 << 16, 4
    b = oracle.Bloom(m, k)
    P = synth.bloom_positions(synth.write_keys(3000, seed=1), m, k)
    for p in P:
        assert b.insert(p) == 0
    assert all(b.contains(p) for p in P)


def test_false_positive_rate_matches_formula():
    # (1 - e^{-kN/m})^k; at m = 2^16, k = 4, N = 8000 that is about 0.0222.
    m, k, N, Q = 1 << 16, 4, 8000, 20000
    b = oracle.Bloom(m, k)
    for p in synth.bloom_positions(synth.write_keys(N, seed=2), m, k):
        b.insert(p)
    probes = synth.bloom_positions(synth.write_keys(Q, seed=3), m, k)
    fp = sum(b.contains(p) for p in probes)
    p = (1.0 - math.exp(-k * N / m)) ** k
    sd = math.sqrt(Q * p * (1 - p))
    assert abs(fp - Q * p) < 3.3 * sd, (fp, Q * p)


def test_global_vector_bits():
    m, k = 256, 2
    b = oracle.Bloom(m, k)
    b.insert([0, 65])
    b.insert([255, 65])
    g = b.get()
    assert g[0] == 1 and g[1] == 2 and g[2] == 0 and g[3] == np.uint64(1 << 63)


def test_window_of_deltas_drops_old_writes():
    # window 2, 3 writes per delta: writes 1-3 fill delta A, 4-6 delta B; write 7
    # opens a new delta in place of A, so writes 1-3 leave the global vector.
    m, k = 512, 1
    b = oracle.Bloom(m, k, window=2, writes_per_delta=3)
    for i in range(1, 7):
        b.insert([i])
    assert [b.contains([i]) for i in range(1, 7)] == [True] * 6
    b.insert([7])
    assert [b.contains([i]) for i in range(1, 8)] == [False] * 3 + [True] * 4
    b.insert([8])
    b.insert([9])
    assert [b.contains([i]) for i in range(1, 10)] == [False] * 3 + [True] * 6
    b.insert([10])  # replaces the delta holding 4-6
    assert [b.contains([i]) for i in range(1, 11)] == [False] * 6 + [True] * 4


def test_or_vector_is_one_write():
    m, k = 200, 3
    b = oracle.Bloom(m, k, window=2, writes_per_delta=1)
    v = np.zeros(4, dtype=np.uint64)
    v[0] = np.uint64(0b1011)
    v[3] = np.uint64(1) << np.uint64(63)    # bit 255 >= m: ignored
    b.or_vector(v)
    g = b.get()
    assert g[0] == 0b1011 and g[3] == 0
    b.insert([5, 6, 7])  # second write: the vector's delta survives (window 2)
    assert b.contains([0, 1, 3])
    b.insert([8, 9, 10])  # third write: the vector's delta is dropped
    assert not b.contains([0, 1, 3]) and b.contains([5, 6, 7])


def test_invalid_position_rejected():
    b = oracle.Bloom(100, 2)
    assert b.insert([5, 100]) == oracle.EINVAL
    assert not b.get().any()


def test_delta_accessor_partitions_the_window():
    """The deltas of the window OR to the global interest vector, the current
    delta holds exactly the latest writes, and ages outside the window fail."""
    import pytest
    from paper_2001_08250_gb300 import synth
    m, k, window, per = 4096, 3, 4, 5
    b = oracle.Bloom(m, k, window, per)
    keys = synth.write_keys(13, seed=31)
    pos = synth.bloom_positions(keys, m, k)
    for p in pos:
        assert b.insert(p) == 0
    acc = np.zeros((m + 63) // 64, dtype=np.uint64)
    for age in range(1, window + 1):
        acc |= b.delta(age)
    assert np.array_equal(acc, b.get())
    # 13 writes, 5 per delta: the current delta holds writes 10..12
    cur = b.delta(1)
    exp = np.zeros_like(cur)
    for p in pos[10:]:
        for q in p:
            exp[int(q) // 64] |= np.uint64(1) << np.uint64(int(q) % 64)
    assert np.array_equal(cur, exp)
    with pytest.raises(ValueError):
        b.delta(window + 1)
