"""Pins of the oracle's serialized-PIR masks (Section 6, steps 6-9).

The paper leaves the PRNG that expands a client seed p_i into the one-time
mask P_i open; the reading taken is the ChaCha20 keystream of RFC 8439 (key
p_i, all-zero nonce, blocks from 0).  The oracle's block function is pinned to
the RFC's published vectors and to an independent library implementation; the
protocol identity of Section 6 (leader XOR of masked responses, client removal
of the masks) is checked on the plain-PIR shape."""

import os
import struct

import numpy as np
import pytest

import oracle
from paper_2001_08250_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "chacha20_rfc8439.txt")


def _vectors():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        key, ctr, nonce, block = line.split()
        out.append((bytes.fromhex(key), int(ctr), bytes.fromhex(nonce), bytes.fromhex(block)))
    return out


def test_rfc8439_block_vectors():
    vecs = _vectors()
    assert len(vecs) == 3
    for key, ctr, nonce, block in vecs:
        assert oracle.chacha20_block(key, ctr, nonce) == block


def test_block_function_matches_library_chacha20():
    algos = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(11)
    for _ in range(40):
        key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
        nonce = rng.integers(0, 256, 12, dtype=np.uint8).tobytes()
        ctr = int(rng.integers(0, 1 << 32))
        enc = algos.Cipher(algos.algorithms.ChaCha20(key, struct.pack("<I", ctr) + nonce),
                           mode=None).encryptor()
        assert oracle.chacha20_block(key, ctr, nonce) == enc.update(bytes(64))


def test_mask_is_the_zero_nonce_keystream_from_block_zero():
    algos = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    seeds = synth.mask_seeds(5, seed=2)
    for s in seeds:
        key = s.tobytes()
        enc = algos.Cipher(algos.algorithms.ChaCha20(key, bytes(16)), mode=None).encryptor()
        ks = np.frombuffer(enc.update(bytes(4096 + 48)), dtype=np.uint8)
        for nbytes in (16, 64, 80, 1024, 4096 + 48):
            assert np.array_equal(oracle.mask(s, nbytes), ks[:nbytes])


def test_mask_prefix_and_seed_dependence():
    s = synth.mask_seeds(3, seed=4)
    long = oracle.mask(s[0], 8192)
    for nbytes in (16, 48, 64, 4080, 4096):
        assert np.array_equal(oracle.mask(s[0], nbytes), long[:nbytes])
    assert not np.array_equal(oracle.mask(s[1], 4096), long[:4096])
    # a one-bit change of the seed changes about half the mask bits
    t = s[0].copy()
    t[31] ^= 0x80
    flips = np.unpackbits(oracle.mask(t, 4096) ^ long[:4096]).mean()
    assert 0.45 < flips < 0.55
    # keystream bits are balanced (4 sigma over 2^16 bits: 0.0078)
    assert abs(np.unpackbits(long).mean() - 0.5) < 0.008


def test_masked_response_without_mask_is_the_plain_answer():
    n, d, z = 100, 2, 64
    T = synth.table_bytes(n, d, z, seed=5).reshape(n, d * z)
    R = synth.random_bits(4, n, seed=5)
    seeds = synth.mask_seeds(4, seed=5)
    masked = oracle.read_batch_masked(T, n, d, z, R, seeds)
    plain = oracle.read_batch(T, n, d, z, R)
    for b in range(4):
        assert np.array_equal(masked[b] ^ oracle.mask(seeds[b], d * z), plain[b])
    # the mask hides the answer: a zero request gives the bare mask
    zero = np.zeros_like(R)
    assert np.array_equal(oracle.read_batch_masked(T, n, d, z, zero, seeds)[2],
                          oracle.mask(seeds[2], d * z))


def test_serialized_pir_leader_combine_recovers_the_bucket():
    """Section 6 steps 1-9 with l = 3 servers on the plain-PIR shape: each
    server answers its share masked by its own seed; the leader XORs the three
    masked responses; the client XORs the three masks off and holds bucket t."""
    n, d, z, l = 1024, 4, 1024, 3
    T = synth.table_bytes(n, d, z, seed=6).reshape(n, d * z)
    tg = synth.targets(16, n, seed=6)
    Q = synth.xor_shares(n, tg, l, seed=6)                      # [16, 3, words]
    seeds = [synth.mask_seeds(16, seed=6, server=i) for i in range(l)]
    masked = [oracle.read_batch_masked(T, n, d, z, Q[:, i, :], seeds[i]) for i in range(l)]
    for q in range(16):
        leader = oracle.reconstruct(np.stack([masked[i][q] for i in range(l)]))
        # no single masked response equals the bucket
        assert not any(np.array_equal(masked[i][q], T[tg[q]]) for i in range(l))
        client = leader.copy()
        for i in range(l):
            client ^= oracle.mask(seeds[i][q], d * z)
        assert np.array_equal(client, T[tg[q]])
