"""The paper-style multi-core CPU engine (a reported baseline of the
benchmark, Section 9.2's CPU server) against the oracle: the same replies for
ragged shapes and thread counts, including more threads than 64-bucket blocks."""

import numpy as np
import pytest

import oracle
from paper_2001_08250_gb300 import synth


@pytest.mark.parametrize("n,d,z,B,threads", [
    (1, 1, 16, 1, 1),
    (63, 2, 16, 5, 3),
    (200, 4, 64, 17, 8),
    (1000, 3, 32, 33, 16),
    (130, 1, 48, 8, 64),
])
def test_engine_matches_oracle(n, d, z, B, threads):
    T = synth.table_bytes(n, d, z, seed=41)
    R = synth.random_bits(B, n, seed=42)
    R[:, -1] |= np.uint64(1) << np.uint64(63)   # bits past n are ignored
    exp = oracle.read_batch(T, n, d, z, R)
    got = oracle.engine_read_batch(T, n, d, z, R, threads=threads)
    assert np.array_equal(got, exp)


def test_engine_three_share_recombination():
    n, d, z = 500, 4, 32
    T = synth.table_bytes(n, d, z, seed=43)
    tg = synth.targets(6, n, seed=44)
    shares = synth.xor_shares(n, tg, 3, seed=45)   # (targets, servers, words)
    for i, t in enumerate(tg):
        rep = oracle.engine_read_batch(T, n, d, z, shares[i], threads=4)
        assert np.array_equal(np.bitwise_xor.reduce(rep, axis=0),
                              T.reshape(n, d * z)[t])
