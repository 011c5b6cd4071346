"""Seeded synthetic inputs for the Talek server read path.

This module only *generates inputs*: table payload bytes, request bit vectors
(and the client-side XOR shares of a one-hot request), bucket pairs and
messages for writes, Bloom-filter bit positions, Poisson arrival times and the
shapes of the uneven multi-table workload.  It holds none of the server-side
arithmetic of the method (no XOR accumulation over buckets, no cuckoo
placement, no Bloom OR); the CPU oracle and the CUDA library each implement
that on their own.  Both sides read their inputs from here, and nothing here
imports either of them.

Randomness.  Every value comes from splitmix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: output ``i`` of the stream keyed by ``key`` is
``mix64(key + (i + 1) * GAMMA)``, which equals the ``i``-th output of the
sequential generator seeded with ``key``.  Streams are keyed by
``stream_key(workload, table, purpose, ...)`` so that every array is
reproducible on its own.

Payloads are uniform random bytes: Talek's stored messages are fixed-size
ciphertexts (Section 5.3, Enc(seqNo | M)), which look uniform to the server.
"""

from __future__ import annotations

import math

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB

# purpose tags for stream_key()
P_TABLE = 1
P_BITS = 2
P_SHARE = 3
P_TARGET = 4
P_KEYS = 5
P_MSG = 6
P_BLOOM = 7
P_ARRIVAL = 8
P_SHAPES = 9
P_MIX = 10
P_SEED = 11

# fixed hash salts used to turn a 64-bit write key into its two buckets and
# its Bloom positions (stand-ins for the client's PRF and cryptographic hashes)
S1 = 0x5EED0001C0C0A001
S2 = 0x5EED0002C0C0A002
SA = 0x5EED0003B100F001
SB = 0x5EED0004B100F002


def mix64_scalar(z: int) -> int:
    z &= M64
    z = ((z ^ (z >> 30)) * _C1) & M64
    z = ((z ^ (z >> 27)) * _C2) & M64
    return z ^ (z >> 31)


def mix64(z: np.ndarray) -> np.ndarray:
    """splitmix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    z ^= z >> np.uint64(30)
    z *= np.uint64(_C1)
    z ^= z >> np.uint64(27)
    z *= np.uint64(_C2)
    z ^= z >> np.uint64(31)
    return z


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    """The first ``count`` outputs of the sequential generator seeded with ``seed``."""
    out, s = [], seed & M64
    for _ in range(count):
        s = (s + GAMMA) & M64
        out.append(mix64_scalar(s))
    return out


def stream_key(*parts: int) -> int:
    h = 0x243F6A8885A308D3
    for p in parts:
        h = mix64_scalar(h ^ (int(p) & M64))
    return h


def stream(key: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the counter-based stream ``key``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    idx *= np.uint64(GAMMA)
    idx += np.uint64(key & M64)
    return mix64(idx)


def _signed(x: int) -> int:
    x &= M64
    return x - (1 << 64) if x >> 63 else x


def stream_torch(key: int, count: int, start: int = 0, device="cuda"):
    """The same outputs as ``stream`` computed with torch int64 tensors on
    ``device`` (two's-complement wrapping arithmetic; logical right shifts
    done as arithmetic shifts masked to the low bits), for inputs too large
    to generate quickly on the host.  Returns an int64 tensor holding the
    uint64 bit patterns."""
    import torch
    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = idx * _signed(GAMMA) + _signed(key)

    def shr(x, s):
        return (x >> s) & ((1 << (64 - s)) - 1)

    z = (z ^ shr(z, 30)) * _signed(_C1)
    z = (z ^ shr(z, 27)) * _signed(_C2)
    return z ^ shr(z, 31)


def table_bytes_torch(n: int, d: int, msg_bytes: int, seed: int = 0, table: int = 0,
                      device="cuda"):
    """``table_bytes`` generated on ``device``: a uint8 tensor [n, d*msg_bytes]
    with the same bytes."""
    import torch
    W = d * msg_bytes
    assert W % 8 == 0
    total = n * W // 8
    out = torch.empty(total, dtype=torch.int64, device=device)
    key = stream_key(seed, table, P_TABLE)
    chunk = 1 << 26
    for s0 in range(0, total, chunk):
        c = min(chunk, total - s0)
        out[s0:s0 + c] = stream_torch(key, c, s0, device)
    return out.view(torch.uint8).view(n, W)


def words_per_row(n: int) -> int:
    """u64 words in one packed request row of ``n`` bits (LSB-first)."""
    return (n + 63) // 64


# --------------------------------------------------------------------------
# table payload
# --------------------------------------------------------------------------

def table_bytes(n: int, d: int, msg_bytes: int, seed: int = 0, table: int = 0,
                out: np.ndarray | None = None) -> np.ndarray:
    """Uniform random table ``T[n][d*msg_bytes]`` (uint8), generated in chunks."""
    W = d * msg_bytes
    assert W % 8 == 0
    total = n * W // 8
    if out is None:
        out = np.empty((n, W), dtype=np.uint8)
    flat = out.reshape(-1).view(np.uint64)
    key = stream_key(seed, table, P_TABLE)
    chunk = 1 << 22
    for s in range(0, total, chunk):
        c = min(chunk, total - s)
        flat[s:s + c] = stream(key, c, s)
    return out


def messages(count: int, msg_bytes: int, seed: int, table: int = 0) -> np.ndarray:
    """``count`` uniform random messages of ``msg_bytes`` bytes."""
    assert msg_bytes % 8 == 0
    w = stream(stream_key(seed, table, P_MSG), count * msg_bytes // 8)
    return w.view(np.uint8).reshape(count, msg_bytes).copy()


# --------------------------------------------------------------------------
# request vectors
# --------------------------------------------------------------------------

def random_bits(rows: int, n: int, seed: int, table: int = 0, purpose: int = P_BITS) -> np.ndarray:
    """``rows`` i.i.d. Bernoulli(0.5) request vectors, packed LSB-first in u64
    words (bit k of a row is bit k%64 of word k//64).  The padding bits at
    positions >= n are random too: the method ignores them."""
    w = words_per_row(n)
    return stream(stream_key(seed, table, purpose), rows * w).reshape(rows, w)


def one_hot(n: int, t: int) -> np.ndarray:
    q = np.zeros(words_per_row(n), dtype=np.uint64)
    q[t >> 6] = np.uint64(1) << np.uint64(t & 63)
    return q


def targets(count: int, n: int, seed: int, table: int = 0) -> np.ndarray:
    """Uniform target buckets in [0, n)."""
    return (stream(stream_key(seed, table, P_TARGET), count) % np.uint64(n)).astype(np.int64)


def xor_shares(n: int, tgts: np.ndarray, l: int, seed: int, table: int = 0) -> np.ndarray:
    """Client-side IT-PIR request splitting (Section 2, steps 1-3): for each
    target t, l-1 uniformly random n-bit vectors q_1..q_{l-1} and the last one
    q_l = e_t XOR q_1 XOR ... XOR q_{l-1}.  Returns uint64 [len(tgts), l, words]."""
    w = words_per_row(n)
    T = len(tgts)
    r = random_bits(T * (l - 1), n, seed, table, P_SHARE).reshape(T, l - 1, w)
    out = np.empty((T, l, w), dtype=np.uint64)
    out[:, :l - 1, :] = r
    last = np.zeros((T, w), dtype=np.uint64)
    for i, t in enumerate(tgts):
        last[i] = one_hot(n, int(t))
    for j in range(l - 1):
        last ^= r[:, j, :]
    out[:, l - 1, :] = last
    return out


def mask_seeds(count: int, seed: int, table: int = 0, server: int = 0) -> np.ndarray:
    """``count`` client seeds p of 32 uniform random bytes each (Section 6
    step 2), one stream per (table, server); uint8 [count, 32]."""
    w = stream(stream_key(seed, table, P_SEED, server), count * 4)
    return w.view(np.uint8).reshape(count, 32).copy()


# --------------------------------------------------------------------------
# writes: keys, bucket pairs, Bloom positions
# --------------------------------------------------------------------------

def write_keys(count: int, seed: int, table: int = 0) -> np.ndarray:
    return stream(stream_key(seed, table, P_KEYS), count)


def bucket_pairs(keys: np.ndarray, n: int) -> tuple[np.ndarray, np.ndarray]:
    """Stand-in for the client's PRF(k_s1, seqNo), PRF(k_s2, seqNo) (Section 5.3):
    b1 = mix64(key ^ S1) mod n, b2 = mix64(key ^ S2) mod n."""
    b1 = mix64(keys ^ np.uint64(S1)) % np.uint64(n)
    b2 = mix64(keys ^ np.uint64(S2)) % np.uint64(n)
    return b1.astype(np.uint64), b2.astype(np.uint64)


def bloom_positions(keys: np.ndarray, m: int, k: int) -> np.ndarray:
    """Stand-in for the client's interest-vector hashes (Section 7): double
    hashing p_i = (h1 + i*h2) mod m with h1 = mix64(key^SA), h2 = mix64(key^SB)|1.
    Returns uint64 [len(keys), k]."""
    h1 = mix64(keys ^ np.uint64(SA))
    h2 = mix64(keys ^ np.uint64(SB)) | np.uint64(1)
    out = np.empty((len(keys), k), dtype=np.uint64)
    for i in range(k):
        out[:, i] = (h1 + np.uint64(i) * h2) % np.uint64(m)
    return out


# --------------------------------------------------------------------------
# arrivals and workload shapes
# --------------------------------------------------------------------------

def uniform01(count: int, key: int) -> np.ndarray:
    """Uniform doubles in (0, 1) from the top 53 bits of the stream."""
    w = stream(key, count) >> np.uint64(11)
    return (w.astype(np.float64) + 0.5) / float(1 << 53)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Open-loop Poisson arrival times (seconds from 0) for ``count`` requests."""
    u = uniform01(count, stream_key(seed, int(rate), P_ARRIVAL))
    return np.cumsum(-np.log(u) / rate)


def op_mix(count: int, write_fraction: float, seed: int) -> np.ndarray:
    """Boolean mask: True where the arriving op is a write."""
    return uniform01(count, stream_key(seed, P_MIX)) < write_fraction


def multi_table_shapes(count: int = 64, seed: int = 3) -> list[tuple[int, int, int, int]]:
    """Uneven multi-table workload: n = floor(2^U(10,17)) buckets, d in {2,4,8},
    message bytes in {256,1024,4096}, reads uniform in 16..512.
    Returns [(n, d, msg_bytes, reads)]."""
    u = uniform01(4 * count, stream_key(seed, P_SHAPES)).reshape(count, 4)
    shapes = []
    for i in range(count):
        n = int(math.floor(2.0 ** (10.0 + 7.0 * u[i, 0])))
        d = (2, 4, 8)[min(2, int(u[i, 1] * 3))]
        z = (256, 1024, 4096)[min(2, int(u[i, 2] * 3))]
        reads = 16 + min(496, int(u[i, 3] * 497))
        shapes.append((n, d, z, reads))
    return shapes
