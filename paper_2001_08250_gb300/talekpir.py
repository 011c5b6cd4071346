"""Thin ctypes binding of libtalekpir (include/talekpir.h).

Argument marshalling only: every step of a read, write or interest-vector
update runs in the library's CUDA kernels.  Host buffers are numpy arrays;
device buffers are torch CUDA tensors (or raw device pointers); streams are
torch.cuda.Stream objects (or raw cudaStream_t values).  If the library is not
built the import of this module's functions raises: there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, EFULL, EAGAIN, ETIMEDOUT, ECUDA, ESHUTDOWN = 0, -1, -2, -3, -4, -5, -6, -7
MAX_JOBS = 128

_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64


class TpirError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {strerror(status)} ({status})" if what else strerror(status))


class ReadJob(ctypes.Structure):
    _fields_ = [("db", _vp), ("B", _u32), ("d_req_bits", _vp), ("d_out", _vp), ("d_seeds", _vp)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _u64), ("max_batch", _u32), ("max_inflight", _u32),
                ("queue_capacity", _u32), ("tick_us", _u32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("lw_log2", _u32), ("warps_b", _u32), ("warps_w", _u32), ("warps_k", _u32),
                ("stage_rows", _u32), ("tile_b", _u32), ("tile_w", _u32), ("candidates", _u32),
                ("us_per_launch", ctypes.c_double), ("lop3_tops", ctypes.c_double),
                ("kernel", _u32), ("tensor_mode", _u32), ("tensor_kc_rows", _u32),
                ("tensor_loads", _u32), ("tensor_candidates", _u32), ("us_lop3", ctypes.c_double),
                ("us_tensor", ctypes.c_double), ("us_m4rm", ctypes.c_double),
                ("us_plain", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Completion(ctypes.Structure):
    _fields_ = [("tag", _u64), ("status", _i32), ("kind", _u32), ("table_id", _u32),
                ("evictions", _u32), ("epoch", _u64), ("t_arrive_ns", _i64),
                ("t_launch_ns", _i64), ("t_done_ns", _i64)]


class Stats(ctypes.Structure):
    _fields_ = [("reads_done", _u64), ("writes_done", _u64), ("rejected", _u64),
                ("failed", _u64), ("launches", _u64), ("reads_per_s", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_batch", ctypes.c_double),
                ("hbm_bytes_in_use", _u64), ("eviction_hist", _u64 * 8),
                ("kernel_launches", _u64 * 6)]


# (name, restype, argtypes) for every entry point of include/talekpir.h
_SIGS = [
    ("tpir_version", ctypes.c_char_p, []),
    ("tpir_last_error", ctypes.c_int, []),
    ("tpir_strerror", ctypes.c_char_p, [ctypes.c_int]),
    ("tpir_db_create", _vp, [_u64, _u32, _u32]),
    ("tpir_db_destroy", None, [_vp]),
    ("tpir_db_create_shard", _vp, [_u64, _u64, _u64, _u32, _u32]),
    ("tpir_bloom_get_compressed", ctypes.c_int, [_vp, _u32, ctypes.c_int32, _vp, _u64, _vp, _vp, _vp]),
    ("tpir_rice_encode_async", ctypes.c_int, [_vp, _u64, ctypes.c_int32, _vp, _u64, _vp, _vp]),
    ("tpir_db_shard_info", ctypes.c_int, [_vp, _vp, _vp]),
    ("tpir_shard_plan", ctypes.c_int, [_u64, _u32, _u32, _vp, _vp]),
    ("tpir_db_info", ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    ("tpir_db_set_policy", ctypes.c_int, [_vp, _u64, _u32, _u64]),
    ("tpir_db_sync", ctypes.c_int, [_vp]),
    ("tpir_db_load", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("tpir_db_load_async", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    ("tpir_db_dump", ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    ("tpir_write", ctypes.c_int, [_vp, _u64, _u64, _vp, _vp]),
    ("tpir_write_batch", ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    ("tpir_write_noalloc", ctypes.c_int, [_vp, _u64, _u64, _vp, _vp, _vp]),
    ("tpir_read_batch", ctypes.c_int, [_vp, _vp, _u32, _vp]),
    ("tpir_read_batch_async", ctypes.c_int, [_vp, _vp, _u32, _vp, _vp]),
    ("tpir_read_batch_masked", ctypes.c_int, [_vp, _vp, _u32, _vp, _vp]),
    ("tpir_read_batch_pipelined", ctypes.c_int, [_vp, _vp, _u64, _u32, _vp]),
    ("tpir_read_batch_masked_async", ctypes.c_int, [_vp, _vp, _u32, _vp, _vp, _vp]),
    ("tpir_mask_generate", ctypes.c_int, [_vp, _u32, _u64, _vp, _vp]),
    ("tpir_xor_combine", ctypes.c_int, [_vp, _u32, _u64, _vp, _vp]),
    ("tpir_db_set_kernel", ctypes.c_int, [_vp, ctypes.c_int]),
    ("tpir_read_multi_async", ctypes.c_int, [_vp, _u32, _vp]),
    ("tpir_autotune", ctypes.c_int, [_vp, _u32, _u32, _vp]),
    ("tpir_tune_save", ctypes.c_int, [ctypes.c_char_p]),
    ("tpir_tune_load", ctypes.c_int, [ctypes.c_char_p]),
    ("tpir_tune_clear", ctypes.c_int, []),
    ("tpir_read_multi_graph_create", ctypes.c_int, [_vp, _u32, _vp]),
    ("tpir_graph_launch", ctypes.c_int, [_vp, _vp]),
    ("tpir_graph_destroy", None, [_vp]),
    ("tpir_selftest_wait_timeout", ctypes.c_int, [_u32]),
    ("tpir_device_status", ctypes.c_int, []),
    ("tpir_kernel_launches", ctypes.c_uint64, []),
    ("tpir_bloom_create", ctypes.c_int, [_vp, _u64, _u32, _u32, _u32]),
    ("tpir_bloom_insert", ctypes.c_int, [_vp, _vp]),
    ("tpir_bloom_insert_batch", ctypes.c_int, [_vp, _vp, _u32]),
    ("tpir_bloom_or_vector", ctypes.c_int, [_vp, _vp]),
    ("tpir_bloom_get", ctypes.c_int, [_vp, _vp]),
    ("tpir_serve_create", ctypes.c_int, [_vp, _vp]),
    ("tpir_serve_add_table", ctypes.c_int, [_vp, _u64, _u32, _u32, _vp]),
    ("tpir_serve_table", ctypes.c_int, [_vp, _u32, _vp]),
    ("tpir_serve_submit_read", ctypes.c_int, [_vp, _u32, _vp, _vp, _u64, _i64]),
    ("tpir_serve_submit_write", ctypes.c_int, [_vp, _u32, _u64, _u64, _vp, _vp, _u64, _i64]),
    ("tpir_serve_poll", ctypes.c_int, [_vp, _vp, _u32, _vp]),
    ("tpir_serve_drain", ctypes.c_int, [_vp]),
    ("tpir_serve_stats", ctypes.c_int, [_vp, _vp]),
    ("tpir_serve_reset_stats", ctypes.c_int, [_vp]),
    ("tpir_serve_destroy", ctypes.c_int, [_vp]),
]

_lib = None


def lib(path: str | None = None):
    """Load libtalekpir.so (building it first if the sources changed)."""
    global _lib
    if _lib is None:
        # TALEKPIR_LIB selects a prebuilt library (e.g. another build variant)
        p = path or os.environ.get("TALEKPIR_LIB") or _build.build()
        if not os.path.exists(p):
            raise RuntimeError(f"libtalekpir not found at {p}")
        L = ctypes.CDLL(p)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().tpir_strerror(status).decode()


def version() -> str:
    return lib().tpir_version().decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise TpirError(rc, what)


def _hptr(a: np.ndarray) -> int:
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _dptr(x) -> int:
    """Device pointer of a torch CUDA tensor, or a raw integer pointer."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


def device_status() -> int:
    return lib().tpir_device_status()


def kernel_launches() -> int:
    """Kernel launches the library has enqueued in this process so far."""
    return int(lib().tpir_kernel_launches())


class DB:
    """One server's blocked cuckoo table of n buckets x d slots x msg_bytes."""

    def __init__(self, n: int, d: int, msg_bytes: int, shard=None):
        """shard = (n_total, row_begin): this db holds buckets [row_begin,
        row_begin + n) of a logical table of n_total buckets, and its reads
        take full-length request rows (ceil(n_total/64) words)."""
        self.n, self.d, self.msg_bytes = int(n), int(d), int(msg_bytes)
        self.row_bytes = self.d * self.msg_bytes
        if shard is None:
            self.n_total, self.row_begin = self.n, 0
            h = lib().tpir_db_create(self.n, self.d, self.msg_bytes)
        else:
            self.n_total, self.row_begin = int(shard[0]), int(shard[1])
            h = lib().tpir_db_create_shard(self.n_total, self.row_begin, self.n, self.d,
                                           self.msg_bytes)
        self.words64 = (self.n_total + 63) // 64
        if not h:
            raise TpirError(lib().tpir_last_error(), "tpir_db_create")
        self.h = h

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().tpir_db_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- state ---------------------------------------------------------------
    @property
    def epoch(self) -> int:
        e = _u64()
        _check(lib().tpir_db_info(self.h, None, None, None, None, ctypes.byref(e)), "tpir_db_info")
        return e.value

    @property
    def table_ptr(self) -> int:
        p = _vp()
        _check(lib().tpir_db_info(self.h, None, None, None, ctypes.byref(p), None), "tpir_db_info")
        return p.value

    def set_policy(self, capacity: int = 0, max_evictions: int = 500, seed: int = 0) -> None:
        _check(lib().tpir_db_set_policy(self.h, capacity, max_evictions, seed), "tpir_db_set_policy")

    def sync(self) -> None:
        """Wait until every write and read submitted on this table has completed."""
        _check(lib().tpir_db_sync(self.h), "tpir_db_sync")

    def set_kernel(self, kernel: int) -> None:
        _check(lib().tpir_db_set_kernel(self.h, kernel), "tpir_db_set_kernel")

    def load(self, table: np.ndarray) -> None:
        t = np.ascontiguousarray(table, dtype=np.uint8)
        _check(lib().tpir_db_load(self.h, _hptr(t), t.nbytes), "tpir_db_load")

    def load_async(self, src, stream=None) -> None:
        """Bulk load from a device tensor (or pinned host tensor) of n*row_bytes bytes."""
        _check(lib().tpir_db_load_async(self.h, src.data_ptr(), src.numel() * src.element_size(),
                                        _stream(stream)), "tpir_db_load_async")

    def dump(self) -> np.ndarray:
        out = np.empty((self.n, self.row_bytes), dtype=np.uint8)
        _check(lib().tpir_db_dump(self.h, _hptr(out), out.nbytes), "tpir_db_dump")
        return out

    # -- writes --------------------------------------------------------------
    def write(self, b1: int, b2: int, msg: np.ndarray) -> tuple[int, int]:
        """Returns (status, evictions); status is OK or EFULL (raises otherwise)."""
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        assert m.size == self.msg_bytes
        ev = _u32()
        rc = lib().tpir_write(self.h, int(b1), int(b2), _hptr(m), ctypes.byref(ev))
        if rc not in (OK, EFULL):
            raise TpirError(rc, "tpir_write")
        return rc, ev.value

    def write_batch(self, b1, b2, msgs) -> tuple[np.ndarray, np.ndarray]:
        b1 = np.ascontiguousarray(b1, dtype=np.uint64)
        b2 = np.ascontiguousarray(b2, dtype=np.uint64)
        msgs = np.ascontiguousarray(msgs, dtype=np.uint8)
        cnt = b1.size
        assert b2.size == cnt and msgs.size == cnt * self.msg_bytes
        st = np.zeros(cnt, dtype=np.int32)
        ev = np.zeros(cnt, dtype=np.uint32)
        _check(lib().tpir_write_batch(self.h, cnt, _hptr(b1), _hptr(b2), _hptr(msgs), _hptr(st),
                                      _hptr(ev)), "tpir_write_batch")
        return st, ev

    # -- reads ---------------------------------------------------------------
    def read_batch(self, req_bits: np.ndarray, out: np.ndarray | None = None) -> np.ndarray:
        """Synchronous read with host buffers: req_bits uint64 [B, words64]."""
        r = np.ascontiguousarray(req_bits, dtype=np.uint64).reshape(-1, self.words64)
        B = r.shape[0]
        if out is None:
            out = np.empty((B, self.row_bytes), dtype=np.uint8)
        assert out.flags["C_CONTIGUOUS"] and out.nbytes == B * self.row_bytes
        _check(lib().tpir_read_batch(self.h, _hptr(r), B, _hptr(out)), "tpir_read_batch")
        return out

    def read_batch_pipelined(self, req_bits: np.ndarray, batch: int,
                             out: np.ndarray | None = None) -> np.ndarray:
        """Synchronous read of many request rows (host) in batches whose copies
        overlap the scans."""
        r = np.ascontiguousarray(req_bits, dtype=np.uint64).reshape(-1, self.words64)
        B = r.shape[0]
        if out is None:
            out = np.empty((B, self.row_bytes), dtype=np.uint8)
        assert out.flags["C_CONTIGUOUS"] and out.nbytes == B * self.row_bytes
        _check(lib().tpir_read_batch_pipelined(self.h, _hptr(r), B, int(batch), _hptr(out)),
               "tpir_read_batch_pipelined")
        return out

    def read_batch_async(self, d_req, B: int, d_out, stream=None) -> None:
        """Asynchronous read with device buffers (torch CUDA tensors or pointers)."""
        _check(lib().tpir_read_batch_async(self.h, _dptr(d_req), int(B), _dptr(d_out),
                                           _stream(stream)), "tpir_read_batch_async")

    def read_batch_masked(self, req_bits: np.ndarray, seeds: np.ndarray,
                          out: np.ndarray | None = None) -> np.ndarray:
        """Serialized-PIR read with host buffers: reply b is masked by the
        ChaCha20 keystream of seeds[b] (uint8 [B, 32])."""
        r = np.ascontiguousarray(req_bits, dtype=np.uint64).reshape(-1, self.words64)
        B = r.shape[0]
        sd = np.ascontiguousarray(seeds, dtype=np.uint8).reshape(B, 32)
        if out is None:
            out = np.empty((B, self.row_bytes), dtype=np.uint8)
        assert out.flags["C_CONTIGUOUS"] and out.nbytes == B * self.row_bytes
        _check(lib().tpir_read_batch_masked(self.h, _hptr(r), B, _hptr(sd), _hptr(out)),
               "tpir_read_batch_masked")
        return out

    def read_batch_masked_async(self, d_req, B: int, d_seeds, d_out, stream=None) -> None:
        """Serialized-PIR read with device buffers (d_seeds: B x 32 bytes)."""
        _check(lib().tpir_read_batch_masked_async(self.h, _dptr(d_req), int(B), _dptr(d_seeds),
                                                  _dptr(d_out), _stream(stream)),
               "tpir_read_batch_masked_async")

    def autotune(self, B: int, reps: int = 3) -> dict:
        """Time every tile shape for B requests on this table; keep the fastest."""
        r = TuneResult()
        _check(lib().tpir_autotune(self.h, int(B), int(reps), ctypes.byref(r)), "tpir_autotune")
        return r.as_dict()

    # -- interest vector -------------------------------------------------------
    def bloom_create(self, m_bits: int, k: int, window: int = 1, writes_per_delta: int = 0) -> None:
        self.bloom_m, self.bloom_k = int(m_bits), int(k)
        _check(lib().tpir_bloom_create(self.h, m_bits, k, window, writes_per_delta), "tpir_bloom_create")

    def bloom_insert(self, positions) -> int:
        p = np.ascontiguousarray(positions, dtype=np.uint64)
        return lib().tpir_bloom_insert(self.h, _hptr(p))

    def bloom_insert_batch(self, positions) -> int:
        p = np.ascontiguousarray(positions, dtype=np.uint64).reshape(-1, self.bloom_k)
        return lib().tpir_bloom_insert_batch(self.h, _hptr(p), p.shape[0])

    def bloom_or_vector(self, vec) -> None:
        v = np.ascontiguousarray(vec, dtype=np.uint64)
        _check(lib().tpir_bloom_or_vector(self.h, _hptr(v)), "tpir_bloom_or_vector")

    def bloom_get_compressed(self, which: int = 0, k: int = -1, cap: int | None = None):
        """Compressed GetUpdates: (stream bytes, nbits, count, k) of the global
        interest vector (which = 0) or of the which-th most recent delta."""
        cap = cap or ((self.bloom_m + 63) // 64) * 8 * 2 + 64
        out = np.zeros(cap, dtype=np.uint8)
        nb, cnt, ku = _u64(), _u64(), _u32()
        _check(lib().tpir_bloom_get_compressed(self.h, int(which), int(k), _hptr(out), cap,
                                               ctypes.byref(nb), ctypes.byref(cnt), ctypes.byref(ku)),
               "tpir_bloom_get_compressed")
        return out[:(nb.value + 7) // 8].copy(), nb.value, cnt.value, ku.value

    def bloom_get(self) -> np.ndarray:
        out = np.empty((self.bloom_m + 63) // 64, dtype=np.uint64)
        _check(lib().tpir_bloom_get(self.h, _hptr(out)), "tpir_bloom_get")
        return out


def tune_save(path: str) -> None:
    _check(lib().tpir_tune_save(path.encode()), "tpir_tune_save")


def tune_load(path: str) -> None:
    _check(lib().tpir_tune_load(path.encode()), "tpir_tune_load")


def tune_clear() -> None:
    _check(lib().tpir_tune_clear(), "tpir_tune_clear")


def rice_encode_async(d_bits, m: int, d_out, cap_bytes: int, d_result, k: int = -1,
                      stream=None) -> None:
    """Rice code of an m-bit device vector into d_out; d_result (3 x uint64
    on the device) receives nbits, count and k."""
    _check(lib().tpir_rice_encode_async(_dptr(d_bits), int(m), int(k), _dptr(d_out), int(cap_bytes),
                                        _dptr(d_result), _stream(stream)), "tpir_rice_encode_async")


def shard_plan(n_total: int, parts: int) -> list[tuple[int, int]]:
    """(row_begin, rows) of each of `parts` row shards of n_total buckets."""
    out = []
    for i in range(parts):
        b, r = _u64(), _u64()
        _check(lib().tpir_shard_plan(int(n_total), int(parts), i, ctypes.byref(b), ctypes.byref(r)),
               "tpir_shard_plan")
        out.append((b.value, r.value))
    return out


def mask_generate(d_seeds, rows: int, nbytes: int, d_out, stream=None) -> None:
    """The one-time masks alone: rows x nbytes keystream bytes into d_out."""
    _check(lib().tpir_mask_generate(_dptr(d_seeds), int(rows), int(nbytes), _dptr(d_out),
                                    _stream(stream)), "tpir_mask_generate")


def xor_combine(d_srcs, nbytes: int, d_dst, stream=None) -> None:
    """The leader's combination: d_dst = XOR of the device buffers d_srcs."""
    arr = (_vp * max(1, len(d_srcs)))(*[_dptr(x) for x in d_srcs])
    _check(lib().tpir_xor_combine(arr, len(d_srcs), int(nbytes), _dptr(d_dst), _stream(stream)),
           "tpir_xor_combine")


def _jobs_array(jobs):
    """jobs: tuples (DB, B, d_req, d_out) or (DB, B, d_req, d_out, d_seeds)."""
    arr = (ReadJob * max(1, len(jobs)))()
    for i, job in enumerate(jobs):
        db, B, d_req, d_out = job[:4]
        arr[i].db = db.h
        arr[i].B = int(B)
        arr[i].d_req_bits = _dptr(d_req)
        arr[i].d_out = _dptr(d_out)
        arr[i].d_seeds = _dptr(job[4]) if len(job) > 4 and job[4] is not None else None
    return arr


def read_multi_async(jobs, stream=None) -> None:
    """jobs: list of (DB, B, d_req, d_out[, d_seeds]) read in one persistent
    launch per kernel kind."""
    _check(lib().tpir_read_multi_async(_jobs_array(jobs), len(jobs), _stream(stream)),
           "tpir_read_multi_async")


class MultiGraph:
    """A many-table read captured once into a CUDA graph; launch() replays it."""

    def __init__(self, jobs):
        self.jobs = jobs  # keep the buffers alive
        h = _vp()
        _check(lib().tpir_read_multi_graph_create(_jobs_array(jobs), len(jobs), ctypes.byref(h)),
               "tpir_read_multi_graph_create")
        self.h = h.value

    def launch(self, stream=None) -> None:
        _check(lib().tpir_graph_launch(self.h, _stream(stream)), "tpir_graph_launch")

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().tpir_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching read/write server over resident tables."""

    def __init__(self, hbm_budget_bytes=0, max_batch=0, max_inflight=0, queue_capacity=0, tick_us=0):
        cfg = ServeConfig(hbm_budget_bytes, max_batch, max_inflight, queue_capacity, tick_us)
        h = _vp()
        _check(lib().tpir_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "tpir_serve_create")
        self.h = h.value
        self.tables = {}

    def add_table(self, n: int, d: int, msg_bytes: int) -> int:
        tid = _u32()
        rc = lib().tpir_serve_add_table(self.h, n, d, msg_bytes, ctypes.byref(tid))
        if rc != OK:
            raise TpirError(rc, "tpir_serve_add_table")
        p = _vp()
        _check(lib().tpir_serve_table(self.h, tid.value, ctypes.byref(p)), "tpir_serve_table")
        db = DB.__new__(DB)
        db.n, db.d, db.msg_bytes = n, d, msg_bytes
        db.row_bytes, db.words64 = d * msg_bytes, (n + 63) // 64
        db.h = p.value
        db.close = lambda: None  # owned by the server
        self.tables[tid.value] = db
        return tid.value

    def table(self, tid: int) -> DB:
        return self.tables[tid]

    def submit_read(self, tid: int, req_bits: np.ndarray, out: np.ndarray, tag: int,
                    t_arrive_ns: int = 0) -> int:
        r = np.ascontiguousarray(req_bits, dtype=np.uint64)
        assert out.flags["C_CONTIGUOUS"]
        return lib().tpir_serve_submit_read(self.h, tid, _hptr(r), _hptr(out), tag, t_arrive_ns)

    def submit_write(self, tid: int, b1: int, b2: int, msg: np.ndarray, tag: int,
                     bloom_positions=None, t_arrive_ns: int = 0) -> int:
        m = np.ascontiguousarray(msg, dtype=np.uint8)
        bp = None if bloom_positions is None else np.ascontiguousarray(bloom_positions, dtype=np.uint64)
        return lib().tpir_serve_submit_write(self.h, tid, int(b1), int(b2), _hptr(m),
                                             None if bp is None else _hptr(bp), tag, t_arrive_ns)

    def poll(self, max_n: int = 4096) -> list:
        arr = (Completion * max_n)()
        nd = _u32()
        _check(lib().tpir_serve_poll(self.h, arr, max_n, ctypes.byref(nd)), "tpir_serve_poll")
        return [arr[i] for i in range(nd.value)]

    def drain(self) -> None:
        _check(lib().tpir_serve_drain(self.h), "tpir_serve_drain")

    def stats(self) -> Stats:
        st = Stats()
        _check(lib().tpir_serve_stats(self.h, ctypes.byref(st)), "tpir_serve_stats")
        return st

    def reset_stats(self) -> None:
        _check(lib().tpir_serve_reset_stats(self.h), "tpir_serve_reset_stats")

    def close(self) -> None:
        if getattr(self, "h", None):
            lib().tpir_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
