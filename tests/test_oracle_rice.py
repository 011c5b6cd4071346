"""Pins of the oracle's compressed interest-vector deltas (Section 7,
GetUpdates): the Golomb-Rice code of the gaps between set bits.

Worked examples written by hand from the definition, an independent decoder
(round trips), the closed-form stream length sum(gap >> k) + count (k + 1),
the parameter rule on exact cases, and the special cases (empty vector,
every bit set, a single far bit, bits past m ignored)."""

import os

import numpy as np
import pytest

import oracle
from paper_2001_08250_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rice_examples.txt")


def _vec(m, positions):
    v = np.zeros((m + 63) // 64, dtype=np.uint64)
    for p in positions:
        v[p // 64] |= np.uint64(1) << np.uint64(p % 64)
    return v


def _stream_bits(out, nbits):
    return "".join(str((int(out[i // 8]) >> (i % 8)) & 1) for i in range(nbits))


def test_hand_worked_examples():
    n = 0
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        m, k, sset, stream = line.split()
        m, k = int(m), int(k)
        pos = [] if sset == "-" else [int(x) for x in sset.split(",")]
        out, nbits, count, kk = oracle.rice_encode(_vec(m, pos), m, k)
        assert kk == k and count == len(pos)
        assert _stream_bits(out, nbits) == ("" if stream == "-" else stream)
        n += 1
    assert n == 5


def test_parameter_rule():
    assert oracle.rice_param(100, 0) == 0
    assert oracle.rice_param(16, 4) == 1      # mean gap 3
    assert oracle.rice_param(8, 8) == 0       # mean gap 0
    assert oracle.rice_param(1 << 20, 1024) == 9   # mean gap 1023
    assert oracle.rice_param(1 << 20, 1023) == 10  # mean gap 1024


def _random_vector(m, density, seed):
    u = synth.uniform01(m, synth.stream_key(seed, 0, 99))
    pos = np.nonzero(u < density)[0]
    return _vec(m, pos.tolist()), pos


@pytest.mark.parametrize("m,density,seed", [(1, 1.0, 1), (64, 0.5, 2), (1000, 0.01, 3),
                                             (4097, 0.3, 4), (1 << 16, 0.001, 5),
                                             (1 << 20, 0.004, 6), (777, 0.0, 7)])
def test_round_trip_and_closed_form_length(m, density, seed):
    v, pos = _random_vector(m, density, seed)
    for k in (None, 0, 3, 12):
        out, nbits, count, kk = oracle.rice_encode(v, m, k)
        assert count == len(pos)
        gaps = np.diff(np.concatenate([[-1], pos])) - 1
        assert nbits == int((gaps >> kk).sum()) + count * (kk + 1)
        assert np.array_equal(oracle.rice_decode(out, nbits, kk, count, m), v)


def test_bits_past_m_are_ignored_and_bad_streams_rejected():
    m = 70
    v = _vec(128, [3, 69, 70, 100])           # 70 and 100 lie past m
    out, nbits, count, k = oracle.rice_encode(v, m, 2)
    assert count == 2
    assert np.array_equal(oracle.rice_decode(out, nbits, k, count, m), _vec(m, [3, 69]))
    with pytest.raises(ValueError):
        oracle.rice_decode(out, nbits - 1, k, count, m)    # truncated
    with pytest.raises(ValueError):
        oracle.rice_decode(out, nbits, k, count, 60)       # position past m


def test_compression_of_sparse_deltas():
    """A delta of N writes x k positions in m bits costs about count (k+2)
    bits: far below m when the delta is sparse (the point of compressing)."""
    m, writes, kpos = 1 << 20, 2000, 4
    keys = synth.write_keys(writes, seed=8)
    pos = np.unique(synth.bloom_positions(keys, m, kpos).reshape(-1))
    v = _vec(m, pos.tolist())
    out, nbits, count, k = oracle.rice_encode(v, m)
    assert count == len(pos)
    assert nbits < count * (k + 3)
    assert len(out) < m // 8 // 10
