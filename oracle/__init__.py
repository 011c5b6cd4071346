"""ctypes loader for the plain-C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the CUDA library; the
library itself never imports it.  See oracle.c for the paper sections each
function follows.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

OK, EINVAL, ENOMEM, EFULL = 0, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (plain C11, -O2)."""
    src = os.path.join(HERE, "oracle.c")
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, src])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.oracle_read.argtypes = [_vp, _u64, _u32, _u32, _vp, _vp]
        L.oracle_read.restype = None
        L.oracle_read_batch.argtypes = [_vp, _u64, _u32, _u32, _vp, _u32, _vp]
        L.oracle_read_batch.restype = None
        L.oracle_reconstruct.argtypes = [_vp, _u32, _u64, _vp]
        L.oracle_reconstruct.restype = None
        L.oracle_splitmix64_next.argtypes = [_u64p]
        L.oracle_splitmix64_next.restype = _u64
        L.oracle_chacha20_block.argtypes = [_vp, _u32, _vp, _vp]
        L.oracle_chacha20_block.restype = None
        L.oracle_mask.argtypes = [_vp, _u64, _vp]
        L.oracle_mask.restype = None
        L.oracle_read_batch_masked.argtypes = [_vp, _u64, _u32, _u32, _vp, _u32, _vp, _vp]
        L.oracle_read_batch_masked.restype = None
        L.oracle_rice_param.argtypes = [_u64, _u64]
        L.oracle_rice_param.restype = _u32
        L.oracle_rice_encode.argtypes = [_vp, _u64, _u32, _vp, _u64, _u64p]
        L.oracle_rice_encode.restype = _u64
        L.oracle_rice_decode.argtypes = [_vp, _u64, _u32, _u64, _u64, _vp]
        L.oracle_rice_decode.restype = ctypes.c_int
        L.oracle_cuckoo_create.argtypes = [_u64, _u32, _u32, _u64, _u32, _u64]
        L.oracle_cuckoo_create.restype = _vp
        L.oracle_cuckoo_destroy.argtypes = [_vp]
        L.oracle_cuckoo_destroy.restype = None
        L.oracle_cuckoo_insert.argtypes = [_vp, _u64, _u64, _vp, _u32p]
        L.oracle_cuckoo_insert.restype = ctypes.c_int
        L.oracle_cuckoo_table.argtypes = [_vp]
        L.oracle_cuckoo_table.restype = _vp
        L.oracle_cuckoo_live.argtypes = [_vp]
        L.oracle_cuckoo_live.restype = _u64
        L.oracle_cuckoo_slot.argtypes = [_vp, _u64, _u64p, _u64p, _u64p]
        L.oracle_cuckoo_slot.restype = ctypes.c_int
        L.oracle_bloom_create.argtypes = [_u64, _u32, _u32, _u32]
        L.oracle_bloom_create.restype = _vp
        L.oracle_bloom_destroy.argtypes = [_vp]
        L.oracle_bloom_destroy.restype = None
        L.oracle_bloom_insert.argtypes = [_vp, _vp]
        L.oracle_bloom_insert.restype = ctypes.c_int
        L.oracle_bloom_or_vector.argtypes = [_vp, _vp]
        L.oracle_bloom_or_vector.restype = None
        L.oracle_bloom_get.argtypes = [_vp, _vp]
        L.oracle_bloom_get.restype = None
        L.oracle_bloom_delta.argtypes = [_vp, _u32, _vp]
        L.oracle_bloom_delta.restype = ctypes.c_int
        L.oracle_bloom_contains.argtypes = [_vp, _vp]
        L.oracle_bloom_contains.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def read(T: np.ndarray, n: int, d: int, z: int, q: np.ndarray) -> np.ndarray:
    """Server answer for one request vector q (u64 words)."""
    T = np.ascontiguousarray(T, dtype=np.uint8)
    q = np.ascontiguousarray(q, dtype=np.uint64)
    assert T.size >= n * d * z and q.size >= (n + 63) // 64
    out = np.empty(d * z, dtype=np.uint8)
    lib().oracle_read(_ptr(T), n, d, z, _ptr(q), _ptr(out))
    return out


def read_batch(T: np.ndarray, n: int, d: int, z: int, R: np.ndarray) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint64).reshape(-1, (n + 63) // 64)
    B = R.shape[0]
    out = np.empty((B, d * z), dtype=np.uint8)
    lib().oracle_read_batch(_ptr(T), n, d, z, _ptr(R), B, _ptr(out))
    return out


def reconstruct(replies: np.ndarray) -> np.ndarray:
    replies = np.ascontiguousarray(replies, dtype=np.uint8)
    l, nbytes = replies.shape
    out = np.empty(nbytes, dtype=np.uint8)
    lib().oracle_reconstruct(_ptr(replies), l, nbytes, _ptr(out))
    return out


def chacha20_block(key: bytes, counter: int, nonce: bytes) -> bytes:
    """RFC 8439 ChaCha20 block function: 64 keystream bytes."""
    assert len(key) == 32 and len(nonce) == 12
    k = np.frombuffer(key, dtype=np.uint8).copy()
    nn = np.frombuffer(nonce, dtype=np.uint8).copy()
    out = np.empty(64, dtype=np.uint8)
    lib().oracle_chacha20_block(_ptr(k), counter, _ptr(nn), _ptr(out))
    return out.tobytes()


def mask(seed, nbytes: int) -> np.ndarray:
    """One-time mask P = PRNG(p) of Section 6 (ChaCha20 keystream, zero nonce)."""
    s = np.ascontiguousarray(np.frombuffer(bytes(seed), dtype=np.uint8) if isinstance(seed, (bytes, bytearray))
                             else seed, dtype=np.uint8)
    assert s.size == 32
    out = np.empty(nbytes, dtype=np.uint8)
    lib().oracle_mask(_ptr(s), nbytes, _ptr(out))
    return out


def read_batch_masked(T: np.ndarray, n: int, d: int, z: int, R: np.ndarray,
                      seeds: np.ndarray) -> np.ndarray:
    """Masked responses R_b XOR PRNG(p_b) of Section 6 step 7."""
    T = np.ascontiguousarray(T, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint64).reshape(-1, (n + 63) // 64)
    B = R.shape[0]
    seeds = np.ascontiguousarray(seeds, dtype=np.uint8).reshape(B, 32)
    out = np.empty((B, d * z), dtype=np.uint8)
    lib().oracle_read_batch_masked(_ptr(T), n, d, z, _ptr(R), B, _ptr(seeds), _ptr(out))
    return out


def rice_param(m: int, count: int) -> int:
    return int(lib().oracle_rice_param(m, count))


def rice_encode(bits: np.ndarray, m: int, k: int | None = None):
    """Rice code of the set bits of an m-bit vector: (stream bytes, nbits,
    count, k); k defaults to rice_param(m, popcount)."""
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    assert b.size >= (m + 63) // 64
    if k is None:
        pc = int(np.unpackbits(b.view(np.uint8), bitorder="little")[:m].sum())
        k = rice_param(m, pc)
    cap = 64
    while True:
        out = np.zeros(cap, dtype=np.uint8)
        cnt = _u64(0)
        nb = int(lib().oracle_rice_encode(_ptr(b), m, k, _ptr(out), cap, ctypes.byref(cnt)))
        if nb != (1 << 64) - 1:
            return out[:(nb + 7) // 8].copy(), nb, int(cnt.value), k
        cap *= 4


def rice_decode(stream: np.ndarray, nbits: int, k: int, count: int, m: int) -> np.ndarray:
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    if s.size == 0:
        s = np.zeros(1, dtype=np.uint8)
    out = np.zeros((m + 63) // 64, dtype=np.uint64)
    rc = lib().oracle_rice_decode(_ptr(s), nbits, k, count, m, _ptr(out))
    if rc != OK:
        raise ValueError("rice stream does not decode")
    return out


def splitmix64(seed: int, count: int) -> list[int]:
    s = _u64(seed)
    return [int(lib().oracle_splitmix64_next(ctypes.byref(s))) for _ in range(count)]


class Cuckoo:
    """Oracle blocked cuckoo table (Section 5.3)."""

    def __init__(self, n, d, z, capacity=0, max_evictions=500, seed=0):
        self.n, self.d, self.z = n, d, z
        self.h = lib().oracle_cuckoo_create(n, d, z, capacity, max_evictions, seed)
        if not self.h:
            raise ValueError("oracle_cuckoo_create failed")

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_cuckoo_destroy(self.h)
            self.h = None

    def insert(self, b1: int, b2: int, msg: np.ndarray) -> tuple[int, int]:
        msg = np.ascontiguousarray(msg, dtype=np.uint8)
        assert msg.size == self.z
        ev = _u32(0)
        rc = lib().oracle_cuckoo_insert(self.h, int(b1), int(b2), _ptr(msg), ctypes.byref(ev))
        return rc, ev.value

    def table(self) -> np.ndarray:
        p = lib().oracle_cuckoo_table(self.h)
        nbytes = self.n * self.d * self.z
        buf = (ctypes.c_uint8 * nbytes).from_address(p)
        return np.frombuffer(buf, dtype=np.uint8).copy().reshape(self.n, self.d * self.z)

    def live(self) -> int:
        return int(lib().oracle_cuckoo_live(self.h))

    def slot(self, s: int):
        b1, b2, seq = _u64(), _u64(), _u64()
        if lib().oracle_cuckoo_slot(self.h, s, ctypes.byref(b1), ctypes.byref(b2), ctypes.byref(seq)):
            return int(b1.value), int(b2.value), int(seq.value)
        return None


class Bloom:
    """Oracle global interest vector with a window of deltas (Section 7)."""

    def __init__(self, m, k, window=1, writes_per_delta=0):
        self.m, self.k = m, k
        self.h = lib().oracle_bloom_create(m, k, window, writes_per_delta)
        if not self.h:
            raise ValueError("oracle_bloom_create failed")

    def __del__(self):
        if getattr(self, "h", None):
            lib().oracle_bloom_destroy(self.h)
            self.h = None

    def insert(self, positions) -> int:
        p = np.ascontiguousarray(positions, dtype=np.uint64)
        assert p.size == self.k
        return lib().oracle_bloom_insert(self.h, _ptr(p))

    def or_vector(self, vec) -> None:
        v = np.ascontiguousarray(vec, dtype=np.uint64)
        assert v.size == (self.m + 63) // 64
        lib().oracle_bloom_or_vector(self.h, _ptr(v))

    def get(self) -> np.ndarray:
        out = np.empty((self.m + 63) // 64, dtype=np.uint64)
        lib().oracle_bloom_get(self.h, _ptr(out))
        return out

    def delta(self, age: int) -> np.ndarray:
        """The age-th most recent delta (1 = current)."""
        out = np.empty((self.m + 63) // 64, dtype=np.uint64)
        if lib().oracle_bloom_delta(self.h, age, _ptr(out)) != OK:
            raise ValueError("no such delta")
        return out

    def contains(self, positions) -> bool:
        p = np.ascontiguousarray(positions, dtype=np.uint64)
        return bool(lib().oracle_bloom_contains(self.h, _ptr(p)))


# ---- the paper-style multi-core CPU engine (a reported baseline, not an oracle)

ENGINE_PATH = os.path.join(HERE, "libcpuengine.so")
_engine = None


def build_engine(force: bool = False) -> str:
    """Compile cpu_engine.c into libcpuengine.so (gcc -O3, pthreads; portable
    code: no machine-specific flags)."""
    src = os.path.join(HERE, "cpu_engine.c")
    if force or not os.path.exists(ENGINE_PATH) or os.path.getmtime(ENGINE_PATH) < os.path.getmtime(src):
        tmp = ENGINE_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O3", "-fPIC", "-shared", "-pthread", "-o", tmp,
                               src])
        os.replace(tmp, ENGINE_PATH)
    return ENGINE_PATH


def engine_read_batch(T: np.ndarray, n: int, d: int, z: int, R: np.ndarray,
                      threads: int | None = None) -> np.ndarray:
    """Replies to the B request rows of R from the multi-core CPU engine."""
    global _engine
    if _engine is None:
        L = ctypes.CDLL(build_engine())
        L.cpu_engine_read_batch.argtypes = [_vp, _u64, _u64, _vp, _u32, _vp, _u32]
        L.cpu_engine_read_batch.restype = ctypes.c_int
        _engine = L
    T = np.ascontiguousarray(T, dtype=np.uint8)
    R = np.ascontiguousarray(R, dtype=np.uint64)
    B = R.shape[0]
    out = np.empty((B, d * z), dtype=np.uint8)
    th = threads or os.cpu_count() or 1
    rc = _engine.cpu_engine_read_batch(_ptr(T), n, d * z, _ptr(R), B, _ptr(out), th)
    if rc != 0:
        raise RuntimeError("cpu engine failed")
    return out
