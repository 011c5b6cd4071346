"""Pins of the oracle's IT-PIR server answer (Section 2) against facts that do
not come from the oracle itself: the worked three-server example, the one-hot
basis, the zero vector, linearity over XOR, a second way of computing the
all-ones answer, and the l = 3 share recombination."""

import os

import numpy as np
import pytest

import oracle
from paper_2001_08250_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_kv(name):
    kv = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            kv[k.strip()] = v.strip()
    return kv


def _bits_to_words(bits):
    q = np.zeros((len(bits) + 63) // 64, dtype=np.uint64)
    for k, b in enumerate(bits):
        if b:
            q[k >> 6] |= np.uint64(1) << np.uint64(k & 63)
    return q


def test_chor_worked_example():
    g = _golden_kv("chor_example_l3_b3.txt")
    blocks = np.array([bytes.fromhex(g[f"block{i}"]) for i in (1, 2, 3)], dtype=object)
    T = np.frombuffer(b"".join(blocks), dtype=np.uint8).reshape(3, 4)
    replies = []
    for name, rname in (("q1", "R1"), ("q2", "R2"), ("q3", "R3")):
        q = _bits_to_words([int(x) for x in g[name].split()])
        r = oracle.read(T, 3, 1, 4, q)
        assert r.tobytes() == bytes.fromhex(g[rname]), name
        replies.append(r)
    assert oracle.reconstruct(np.stack(replies)).tobytes() == bytes.fromhex(g["B_beta"])
    # the shares recombine to q'
    qs = [np.array([int(x) for x in g[k].split()]) for k in ("q1", "q2", "q3")]
    assert list(qs[0] ^ qs[1] ^ qs[2]) == [int(x) for x in g["q_prime"].split()]


@pytest.mark.parametrize("n,d,z", [(1, 1, 16), (5, 1, 16), (64, 2, 48), (65, 4, 16), (200, 8, 32)])
def test_one_hot_returns_that_bucket(n, d, z):
    T = synth.table_bytes(n, d, z, seed=11, table=n)
    for t in sorted({0, n - 1, min(63, n - 1), min(64, n - 1), n // 2}):
        assert np.array_equal(oracle.read(T, n, d, z, synth.one_hot(n, t)), T[t])


def test_lsb_first_bit_order():
    n, d, z = 130, 1, 16
    T = synth.table_bytes(n, d, z, seed=5)
    q = np.zeros(3, dtype=np.uint64)
    q[0] = np.uint64(0b10)          # bit 1 of word 0 -> bucket 1
    q[2] = np.uint64(1)             # bit 0 of word 2 -> bucket 128
    assert np.array_equal(oracle.read(T, n, d, z, q), T[1] ^ T[128])


def test_zero_vector_returns_zero():
    n, d, z = 300, 4, 64
    T = synth.table_bytes(n, d, z, seed=1)
    assert not oracle.read(T, n, d, z, np.zeros(5, dtype=np.uint64)).any()


def test_padding_bits_ignored():
    n, d, z = 70, 2, 16
    T = synth.table_bytes(n, d, z, seed=2)
    q = synth.random_bits(1, n, seed=3)[0]
    q_clean = q.copy()
    q_clean[1] &= np.uint64((1 << (n - 64)) - 1)
    q_dirty = q_clean.copy()
    q_dirty[1] |= ~np.uint64((1 << (n - 64)) - 1)
    assert np.array_equal(oracle.read(T, n, d, z, q_dirty), oracle.read(T, n, d, z, q_clean))


def test_linearity_over_xor():
    n, d, z = 257, 4, 32
    T = synth.table_bytes(n, d, z, seed=4)
    R = synth.random_bits(20, n, seed=5)
    for i in range(10):
        a, b = R[2 * i], R[2 * i + 1]
        lhs = oracle.read(T, n, d, z, a ^ b)
        rhs = oracle.read(T, n, d, z, a) ^ oracle.read(T, n, d, z, b)
        assert np.array_equal(lhs, rhs)


def test_tiny_exhaustive_basis_and_linearity():
    # On n = 5 every request vector is checked: A(e_t) = T[t] for the basis and
    # A(q ^ q') = A(q) ^ A(q') for all 32 x 32 pairs fix A completely.
    n, d, z = 5, 1, 16
    T = synth.table_bytes(n, d, z, seed=6)
    ans = {}
    for v in range(32):
        ans[v] = oracle.read(T, n, d, z, np.array([v], dtype=np.uint64))
    for t in range(n):
        assert np.array_equal(ans[1 << t], T[t])
    for a in range(32):
        for b in range(32):
            assert np.array_equal(ans[a ^ b], ans[a] ^ ans[b])


def test_all_ones_equals_xor_fold():
    n, d, z = 1000, 4, 64
    T = synth.table_bytes(n, d, z, seed=7)
    q = np.full((n + 63) // 64, np.uint64((1 << 64) - 1), dtype=np.uint64)
    fold = np.bitwise_xor.reduce(T.view(np.uint64), axis=0).view(np.uint8)
    assert np.array_equal(oracle.read(T, n, d, z, q), fold)


def test_three_share_recombination_recovers_target():
    # Section 2 steps 1-6 with l = 3 on the plain-PIR workload shape
    # (n = 1024 buckets, d = 4, 1024-byte messages), 16 targets.
    n, d, z = 1024, 4, 1024
    T = synth.table_bytes(n, d, z, seed=0)
    tg = synth.targets(16, n, seed=0)
    S = synth.xor_shares(n, tg, 3, seed=0)
    for i, t in enumerate(tg):
        replies = oracle.read_batch(T, n, d, z, S[i])
        assert np.array_equal(oracle.reconstruct(replies), T[t])
        # each single share looks nothing like the target (sanity: not one-hot)
        assert all(np.count_nonzero(S[i, j]) > 1 for j in range(3))


def test_batch_matches_single_reads():
    n, d, z = 333, 2, 48
    T = synth.table_bytes(n, d, z, seed=8)
    R = synth.random_bits(7, n, seed=9)
    out = oracle.read_batch(T, n, d, z, R)
    for b in range(7):
        assert np.array_equal(out[b], oracle.read(T, n, d, z, R[b]))


def test_reconstruct_is_xor_of_replies():
    r = np.array([[1, 2, 4, 8], [3, 0, 4, 0], [0, 2, 0, 8]], dtype=np.uint8)
    assert list(oracle.reconstruct(r)) == [2, 0, 0, 0]
