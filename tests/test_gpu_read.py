"""GPU parity of the PIR read kernels against the oracle, through the C ABI.

Replies must be bit-exact.  Small and ragged shapes are compared element by
element on every row; the paper-scale tables are compared on sampled rows and
with a GF(2) Freivalds check of the whole batch, in the launch configuration
the benchmark times."""

import numpy as np
import pytest

import oracle
from gpu_helpers import check_rows, dev_out, freivalds, require_cuda, to_dev, to_host
from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu

PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR = 1, 2, 3, 4, 5


def _db(n, d, z, T):
    db = talekpir.DB(n, d, z)
    db.load(T)
    return db


# n not a multiple of 32/64/stage rows, d = 1..8, msg 16..4096, B around
# the tile edges, padding bits set (random_bits fills whole words)
EDGE = [
    (1, 1, 16, 1), (1, 4, 1024, 5), (63, 1, 16, 3), (64, 2, 48, 9), (65, 4, 16, 31),
    (200, 8, 32, 33), (333, 2, 256, 64), (1000, 1, 4096, 17), (1024, 4, 1024, 257),
    (4097, 2, 256, 40), (777, 3, 80, 12), (130, 8, 4096, 8), (2049, 1, 64, 100),
]


@pytest.mark.parametrize("n,d,z,B", EDGE)
@pytest.mark.parametrize("kernel", [PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR])
def test_edge_shapes_bit_exact(n, d, z, B, kernel):
    require_cuda()
    T = synth.table_bytes(n, d, z, seed=21, table=n * 7 + d)
    R = synth.random_bits(B, n, seed=22, table=n)
    exp = oracle.read_batch(T, n, d, z, R)
    with _db(n, d, z, T) as db:
        db.set_kernel(kernel)
        got = db.read_batch(R)
        assert np.array_equal(got, exp)
        # the asynchronous device-buffer entry point gives the same replies
        dR, dO = to_dev(R), dev_out(B, d * z)
        db.read_batch_async(dR, B, dO)
        assert np.array_equal(to_host(dO), exp)
    assert talekpir.device_status() == talekpir.OK


def test_empty_batch_and_zero_vector():
    require_cuda()
    n, d, z = 100, 2, 64
    T = synth.table_bytes(n, d, z, seed=3)
    with _db(n, d, z, T) as db:
        assert db.read_batch(np.zeros((0, 2), dtype=np.uint64)).shape == (0, d * z)
        for k in (PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR):
            db.set_kernel(k)
            assert not db.read_batch(np.zeros((6, 2), dtype=np.uint64)).any()
            # one-hot rows return exactly their bucket
            R = np.stack([synth.one_hot(n, t) for t in (0, 1, 63, 64, 99)])
            assert np.array_equal(db.read_batch(R), T[[0, 1, 63, 64, 99]])


def test_plain_pir_workload_cuckoo_filled_and_three_shares():
    """n = 1024 buckets, d = 4, 1024-byte messages (4 MiB): filled to load 0.5
    (2048 messages) through the device write path, then 64 reads, each split
    into l = 3 XOR shares; every share's reply matches the oracle and the three
    replies recombine to the target bucket."""
    require_cuda()
    n, d, z = 1024, 4, 1024
    keys = synth.write_keys(2048, seed=0)
    b1, b2 = synth.bucket_pairs(keys, n)
    M = synth.messages(2048, z, seed=0)
    oc = oracle.Cuckoo(n, d, z, 0, 500, seed=0)
    for i in range(2048):
        assert oc.insert(int(b1[i]), int(b2[i]), M[i])[0] == 0
    T = oc.table()
    with talekpir.DB(n, d, z) as db:
        db.set_policy(0, 500, 0)
        st, ev = db.write_batch(b1, b2, M)
        assert (st == 0).all()
        assert np.array_equal(db.dump(), T)
        tg = synth.targets(64, n, seed=0)
        S = synth.xor_shares(n, tg, 3, seed=0).reshape(192, -1)
        for kernel in (PLAIN, BATCHED, M4RM):
            db.set_kernel(kernel)
            got = db.read_batch(S)
            assert np.array_equal(got, oracle.read_batch(T, n, d, z, S))
            rec = got.reshape(64, 3, -1)
            for i, t in enumerate(tg):
                assert np.array_equal(rec[i, 0] ^ rec[i, 1] ^ rec[i, 2], T[t])


@pytest.fixture(scope="module")
def paper_scale():
    n, d, z = 32768, 4, 1024
    T = synth.table_bytes(n, d, z, seed=0)
    return n, d, z, T


@pytest.mark.parametrize("B", [1, 32, 256])
def test_paper_scale_table_batches(paper_scale, B):
    """n = 32768, d = 4, 1 KiB messages (128 MiB), Bernoulli(0.5) requests in
    batches of B, through the device-buffer entry point the benchmark times
    (at B = 256 the CTA-pair tensor-core kernel, the benchmark's launch)."""
    require_cuda()
    n, d, z, T = paper_scale
    R = synth.random_bits(B, n, seed=1, table=B)
    with _db(n, d, z, T) as db:
        dR, dO = to_dev(R), dev_out(B, d * z)
        db.read_batch_async(dR, B, dO)
        Out = to_host(dO)
        # 16 sampled rows (both M-tiles, both CTAs of a pair at B = 256) and 20
        # Freivalds trials at the benchmarked shape
        rows = sorted({0, B - 1, B // 2} | set(np.random.default_rng(B).integers(0, B, 13).tolist()))
        check_rows(T, n, d, z, R, Out, rows)
        freivalds(T, n, d, z, R, Out, trials=20, seed=B)
        # forced kernels agree with the automatic choice
        for k in (PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR):
            db.set_kernel(k)
            dO2 = dev_out(B, d * z)
            db.read_batch_async(dR, B, dO2)
            assert np.array_equal(to_host(dO2), Out)
    assert talekpir.device_status() == talekpir.OK


def test_paper_scale_three_share_recombination(paper_scale):
    require_cuda()
    n, d, z, T = paper_scale
    tg = synth.targets(64, n, seed=5)
    S = synth.xor_shares(n, tg, 3, seed=5).reshape(192, -1)
    with _db(n, d, z, T) as db:
        got = db.read_batch(S).reshape(64, 3, -1)
    for i, t in enumerate(tg):
        assert np.array_equal(got[i, 0] ^ got[i, 1] ^ got[i, 2], T[t])


def test_multi_table_one_launch_bit_exact():
    """Uneven tables (n, d, msg_bytes and B all differ) in one persistent launch."""
    require_cuda()
    shapes = [(1100, 2, 256, 16), (3000, 4, 1024, 40), (513, 8, 4096, 7), (2048, 2, 256, 300),
              (97, 1, 16, 1), (4096, 4, 1024, 129), (700, 8, 256, 64), (64, 2, 4096, 33)]
    dbs, jobs, exp = [], [], []
    for i, (n, d, z, B) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=30, table=i)
        R = synth.random_bits(B, n, seed=31, table=i)
        db = _db(n, d, z, T)
        dbs.append(db)
        dR, dO = to_dev(R), dev_out(B, d * z)
        jobs.append((db, B, dR, dO))
        exp.append(oracle.read_batch(T, n, d, z, R))
    talekpir.read_multi_async(jobs)
    for (db, B, dR, dO), e in zip(jobs, exp):
        assert np.array_equal(to_host(dO), e)
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_multi_table_tensor_launch_chunks_and_request_paths():
    """More tables than one tensor-core launch holds (its parameters carry
    three tensor maps per table, 64 tables per launch): 100 small tables of
    96..299 requests, forced to the tensor-core kernel, with even and odd
    request-word counts (staged as rows and as row pairs) and every third
    request block at an 8-byte offset (per-thread loads instead of TMA
    staging), read in one call and from a captured graph; every reply
    bit-exact."""
    torch = require_cuda()
    rng = np.random.default_rng(90)
    dbs, jobs, exp, keep = [], [], [], []
    for i in range(100):
        n = int(rng.integers(60, 400))
        d, z, B = int(rng.choice([1, 2])), int(rng.choice([32, 64, 256])), int(rng.integers(96, 300))
        T = synth.table_bytes(n, d, z, seed=91, table=i)
        R = synth.random_bits(B, n, seed=92, table=i)
        db = _db(n, d, z, T)
        db.set_kernel(TENSOR)
        dbs.append(db)
        if i % 3 == 0:
            flat = to_dev(np.concatenate([np.zeros(1, np.uint64), R.reshape(-1)]))
            keep.append(flat)
            dR = flat[1:]
        else:
            dR = to_dev(R)
        jobs.append((db, B, dR, dev_out(B, d * z)))
        exp.append(oracle.read_batch(T, n, d, z, R))
    talekpir.read_multi_async(jobs)
    for (db, B, dR, dO), e in zip(jobs, exp):
        assert np.array_equal(to_host(dO), e)
    g = talekpir.MultiGraph(jobs)
    for (_, _, _, dO) in jobs:
        dO.fill_(0xA5)
    g.launch()
    torch.cuda.synchronize()
    for (db, B, dR, dO), e in zip(jobs, exp):
        assert np.array_equal(to_host(dO), e)
    g.close()
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_multi_table_graph_replays_see_writes():
    """The many-table read captured into a CUDA graph: replays give the oracle's
    replies, and a replay after a write to one table sees that write."""
    torch = require_cuda()
    shapes = [(1100, 2, 256, 16), (3000, 4, 1024, 40), (700, 8, 256, 64)]
    dbs, jobs, Ts, Rs = [], [], [], []
    for i, (n, d, z, B) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=50, table=i)
        R = synth.random_bits(B, n, seed=51, table=i)
        db = _db(n, d, z, T)
        dbs.append(db)
        Ts.append(T)
        Rs.append(R)
        jobs.append((db, B, to_dev(R), dev_out(B, d * z)))
    g = talekpir.MultiGraph(jobs)
    for rep in range(2):
        for (_, _, _, dO) in jobs:
            dO.zero_()
        g.launch()
        torch.cuda.synchronize()
        for (n, d, z, B), T, R, (_, _, _, dO) in zip(shapes, Ts, Rs, jobs):
            assert np.array_equal(to_host(dO), oracle.read_batch(T, n, d, z, R)), rep
    # a write to table 1, then a replay
    n, d, z, B = shapes[1]
    oc = oracle.Cuckoo(n, d, z, 0, 500, seed=0)
    msg = synth.messages(1, z, seed=52)[0]
    assert dbs[1].write(5, 6, msg)[0] == talekpir.OK   # table was bulk-loaded: every slot free
    oc.insert(5, 6, msg)
    T1 = Ts[1].copy()
    T1[5, :z] = msg
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(to_host(jobs[1][3]), oracle.read_batch(T1, n, d, z, Rs[1]))
    g.close()
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_autotuned_shape_stays_bit_exact():
    """The autotuner times every tile shape on the table; the shape it keeps
    is used by later launches, which must still match the oracle."""
    require_cuda()
    n, d, z, B = 4100, 2, 512, 100
    T = synth.table_bytes(n, d, z, seed=60)
    R = synth.random_bits(B, n, seed=61)
    with _db(n, d, z, T) as db:
        res = db.autotune(B, reps=2)
        assert res["candidates"] >= 2 and res["us_per_launch"] > 0
        assert res["warps_b"] * res["warps_w"] * res["warps_k"] == 8
        db.set_kernel(BATCHED)
        assert np.array_equal(db.read_batch(R), oracle.read_batch(T, n, d, z, R))
    talekpir.tune_clear()


def test_multi_table_large_batches_bit_exact():
    """Many tables with large batches in one call: those on rows of >= 256
    bytes share one launch of the tensor-core kernel (and, with their dbs
    forced to kernel 4, the Four-Russians kernel's 256- and 512-request
    launches), the narrow one goes to the register-tiled kernel; all
    bit-exact, directly and replayed from a captured graph."""
    require_cuda()
    shapes = [(1100, 2, 256, 200), (3000, 4, 1024, 256), (513, 8, 4096, 400), (700, 1, 64, 180),
              (2049, 2, 512, 333), (4096, 4, 1024, 96), (300, 2, 512, 128)]
    dbs, jobs, exp = [], [], []
    for i, (n, d, z, B) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=80, table=i)
        R = synth.random_bits(B, n, seed=81, table=i)
        db = _db(n, d, z, T)
        dbs.append(db)
        jobs.append((db, B, to_dev(R), dev_out(B, d * z)))
        exp.append(oracle.read_batch(T, n, d, z, R))
    for forced in (0, M4RM, TENSOR):
        for db in dbs:
            db.set_kernel(forced)
        for (_, _, _, dO) in jobs:
            dO.zero_()
        talekpir.read_multi_async(jobs)
        for (db, B, dR, dO), e in zip(jobs, exp):
            assert np.array_equal(to_host(dO), e), forced
        g = talekpir.MultiGraph(jobs)
        for (_, _, _, dO) in jobs:
            dO.fill_(0x5A)
        g.launch()
        for (db, B, dR, dO), e in zip(jobs, exp):
            assert np.array_equal(to_host(dO), e), forced
        g.close()
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("n,B,loads,mode", [(32768, 128, 0, 2), (32767, 256, 0, 2), (32768, 256, 0, 3),
                                            (65536, 300, 0, 2), (65536, 200, 1, 2), (32768, 64, 1, 2)])
def test_tensor_kernel_counts_at_the_chunk_bound(n, B, loads, mode, tmp_path):
    """One accumulator over a whole k-chunk of 32 768 buckets: a tuning plan
    (loaded as a user would) makes the tensor-core read take items of whole
    32 768-bucket k-chunks (mode 2: on CTA pairs above 128 requests with
    TMA-staged rows; mode 3: on single CTAs), and all-ones requests then drive
    each count to its largest values: 32 767 (odd: a column set on every row
    but one, or every row of a 32 767-bucket table) and 32 768 (even),
    besides counts of 16 384 and 10 923 (rows k odd, rows k = 0 mod 3).  With
    65 536 buckets two full chunks are XOR-combined.  Every reply bit-exact."""
    require_cuda()
    d, z = 1, 256                       # 64 words: a row width plans may steer
    T = np.zeros((n, d * z), dtype=np.uint8)
    T[1:, 0:4] = 0xFF                   # every row but row 0
    T[:, 4:8] = 0xFF                    # every row
    T[1::2, 8:12] = 0xFF                # odd rows
    T[0::3, 12:16] = 0xFF               # rows 0 mod 3
    T[:, 16:] = synth.table_bytes(n, 1, 240, seed=95)
    R = np.full((B, (n + 63) // 64), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    bclass = max(0, (B - 1).bit_length())
    nclass = max(0, (n - 1).bit_length())
    plan = tmp_path / "plan.json"
    plan.write_text('{"plans": [\n{"row_words": 64, "batch_class": %d, "n_class": %d, "kernel": 5, '
                    '"tensor_mode": %d, "tensor_kc_rows": 32768, "tensor_loads": %d}\n]}\n'
                    % (bclass, nclass, mode, loads))
    talekpir.tune_load(str(plan))
    try:
        exp = oracle.read(T, n, d, z, R[0])
        assert exp[0:4].any() == (((n - 1) % 2) == 1)
        with _db(n, d, z, T) as db:
            got = db.read_batch(R)
        assert (got == exp[None, :]).all()
    finally:
        talekpir.tune_clear()
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("n,B", [(32768, 256), (40003, 129), (70001, 300), (65, 7),
                                 (131075, 64)])
def test_tensor_kernel_exact_counts_all_ones(n, B):
    """All-ones requests against a table whose columns are set on every row,
    on even rows, or on rows k = 0 mod 3: the tensor-core kernel's
    accumulators reach the largest counts a k-chunk can hold (every bucket
    selected), and the three column classes give both parities."""
    require_cuda()
    d, z = 1, 64
    T = np.zeros((n, d * z), dtype=np.uint8)
    T[:, 32:] = 0xFF
    T[0::2, 16:32] = 0xFF
    T[0::3, :16] = 0xA5
    R = np.full((B, (n + 63) // 64), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    exp = oracle.read(T, n, d, z, R[0])
    assert exp.any()
    with _db(n, d, z, T) as db:
        db.set_kernel(TENSOR)
        got = db.read_batch(R)
    assert (got == exp[None, :]).all()
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("n,B", [(1024, 200), (4096, 96), (40000, 257), (4097, 300)])
def test_tensor_kernel_request_rows_staged_or_loaded(n, B):
    """Request rows 16-byte aligned with an even number of words are staged
    into shared memory by TMA; rows at an 8-byte offset (or an odd word
    count, n = 4097) are loaded by the expander threads.  Both give the
    oracle's replies, for batches below, at and past one 256-request block."""
    require_cuda()
    d, z = 2, 256
    T = synth.table_bytes(n, d, z, seed=31, table=n)
    R = synth.random_bits(B, n, seed=32, table=n)
    exp = oracle.read_batch(T, n, d, z, R)
    with _db(n, d, z, T) as db:
        db.set_kernel(TENSOR)
        dO = dev_out(B, d * z)
        dR = to_dev(R)
        db.read_batch_async(dR, B, dO)
        assert np.array_equal(to_host(dO), exp)
        flat = to_dev(np.concatenate([np.zeros(1, np.uint64), R.reshape(-1)]))
        dO.zero_()
        db.read_batch_async(flat[1:], B, dO)  # rows 8 bytes off a 16-byte boundary
        assert np.array_equal(to_host(dO), exp)
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("n,offset", [(4096, 0), (4160, 0), (4096, 1)])
def test_tensor_kernel_back_to_back_launches(n, offset):
    """Thirty launches of the tensor-core kernel back to back on one stream,
    alternating two tables, in each request-staging mode (rows of 64 words
    staged as rows, of 65 words as row pairs, and an 8-byte offset buffer
    read by the expander threads): every reply of every launch bit-exact.
    Catches ring-slot reuse races that a single launch can hide."""
    torch = require_cuda()
    d, z, B = 4, 256, 300
    Ts = [synth.table_bytes(n, d, z, seed=41, table=t) for t in range(2)]
    R = synth.random_bits(B, n, seed=42, table=n)
    exps = [oracle.read_batch(T, n, d, z, R) for T in Ts]
    dbs = [_db(n, d, z, T) for T in Ts]
    for db in dbs:
        db.set_kernel(TENSOR)
    flat = to_dev(np.concatenate([np.zeros(offset, np.uint64), R.reshape(-1)]))
    dR = flat[offset:]
    outs = [dev_out(B, d * z) for _ in range(30)]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for i, o in enumerate(outs):
            dbs[i % 2].read_batch_async(dR, B, o, s)
    s.synchronize()
    for i, o in enumerate(outs):
        assert np.array_equal(to_host(o), exps[i % 2]), f"launch {i}"
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("B_total,batch,kernel", [(1000, 256, 0), (37, 256, 0), (513, 128, TENSOR),
                                                  (300, 7, PLAIN), (257, 64, BATCHED), (600, 200, M4RM)])
def test_pipelined_host_reads_bit_exact(B_total, batch, kernel):
    """The pipelined host-buffer read (copies overlapping the scans over three
    rotating device slots) gives the oracle's replies for every request, with
    a ragged last batch and a batch larger than the request set."""
    torch = require_cuda()
    n, d, z = 3000, 4, 1024
    T = synth.table_bytes(n, d, z, seed=101)
    R = synth.random_bits(B_total, n, seed=102, table=B_total)
    hR = torch.from_numpy(R.view(np.int64)).pin_memory().numpy().view(np.uint64)
    hO = torch.empty((B_total, d * z), dtype=torch.uint8).pin_memory().numpy()
    with _db(n, d, z, T) as db:
        db.set_kernel(kernel)
        got = db.read_batch_pipelined(hR, batch, hO)
        assert np.array_equal(got, oracle.read_batch(T, n, d, z, R))
        # pageable buffers give the same replies (the copies just do not overlap)
        assert np.array_equal(db.read_batch_pipelined(R, batch), got)
    assert talekpir.device_status() == talekpir.OK


def test_pipelined_reads_of_several_tables_from_several_threads():
    """One host thread per table (each thread the only user of its db, as the
    API allows): concurrent pipelined host-buffer reads of three tables of
    different shapes, batches that take the CTA-pair tensor-core kernel, the
    single-CTA one and the plain stream; every reply equals the oracle's."""
    torch = require_cuda()
    from concurrent.futures import ThreadPoolExecutor
    shapes = [(3000, 4, 1024, 700, 256), (2049, 2, 512, 390, 100), (5000, 1, 256, 65, 3)]
    dbs, jobs = [], []
    for i, (n, d, z, Bt, batch) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=120, table=i)
        R = synth.random_bits(Bt, n, seed=121, table=i)
        hR = torch.from_numpy(R.view(np.int64)).pin_memory().numpy().view(np.uint64)
        hO = torch.empty((Bt, d * z), dtype=torch.uint8).pin_memory().numpy()
        db = _db(n, d, z, T)
        dbs.append(db)
        jobs.append((db, hR, hO, batch, oracle.read_batch(T, n, d, z, R)))
    try:
        def run(job):
            db, hR, hO, batch, _ = job
            for _ in range(3):
                db.read_batch_pipelined(hR, batch, hO)
        with ThreadPoolExecutor(len(jobs)) as ex:
            list(ex.map(run, jobs))
        for db, hR, hO, batch, exp in jobs:
            assert np.array_equal(hO, exp), (db.n, batch)
    finally:
        for db in dbs:
            db.close()
    assert talekpir.device_status() == talekpir.OK


def test_kernel_launch_counter_counts_the_reads_launches():
    """tpir_kernel_launches counts every kernel the library enqueues: one
    CTA-pair tensor-core launch for a 256-request read of a table that fits
    one k-chunk, more when replies are initialised first, none for a call
    that launches nothing (B = 0)."""
    require_cuda()
    n, d, z = 4096, 4, 1024
    T = synth.table_bytes(n, d, z, seed=130)
    R = synth.random_bits(256, n, seed=131)
    with _db(n, d, z, T) as db:
        dR, dO = to_dev(R), dev_out(256, d * z)
        db.read_batch_async(dR, 256, dO)      # builds the transposed copy
        db.sync()
        k0 = talekpir.kernel_launches()
        db.read_batch_async(dR, 256, dO)
        db.sync()
        assert talekpir.kernel_launches() - k0 == 1
        k1 = talekpir.kernel_launches()
        db.read_batch_async(dR, 0, dO)
        assert talekpir.kernel_launches() == k1
        assert np.array_equal(to_host(dO), oracle.read_batch(T, n, d, z, R))
    assert talekpir.device_status() == talekpir.OK


# CTA-pair tensor-core form: B just above one M-tile, blocks whose odd CTA has
# no request, odd / even request-word counts (row pairs / rows staged by TMA),
# n below one stage, an odd number of strips (the last pair half past the
# row), tables longer than one 32 768-bucket k-chunk (partials XOR-combined)
PAIR_SHAPES = [(63, 1, 256, 129), (300, 2, 512, 200), (513, 1, 4096, 384), (4096, 4, 256, 511),
               (70001, 1, 448, 130)]


@pytest.mark.parametrize("n,d,z,B", PAIR_SHAPES)
def test_pair_tensor_form_bit_exact(n, d, z, B):
    """Every reply of the tensor-core read on CTA pairs, plain and masked
    (one k-chunk: keystream in the epilogue; several: masks written by the
    reply initialisation), equals the oracle's."""
    require_cuda()
    T = synth.table_bytes(n, d, z, seed=140, table=n)
    R = synth.random_bits(B, n, seed=141, table=n)
    S = synth.mask_seeds(B, seed=142, table=n)
    with _db(n, d, z, T) as db:
        db.set_kernel(TENSOR)
        assert np.array_equal(db.read_batch(R), oracle.read_batch(T, n, d, z, R))
        assert np.array_equal(db.read_batch_masked(R, S), oracle.read_batch_masked(T, n, d, z, R, S))
    assert talekpir.device_status() == talekpir.OK


def test_multi_table_pair_launch_bit_exact():
    """Large batches on tables of >= 8192 buckets share one persistent
    CTA-pair launch per request-staging mode in a many-table call: rows of
    an even word count (TMA rows) and of an odd one (row pairs), a masked job
    (keystream in the epilogue), a table of two k-chunks (partials
    XOR-combined into initialised replies), next to a job of <= 128 requests
    in the single-CTA launch; every reply equals the oracle's, directly and
    replayed from a captured graph."""
    torch = require_cuda()
    shapes = [(8192, 1, 256, 129, False), (9000, 2, 256, 256, False), (16385, 1, 512, 300, False),
              (40000, 1, 256, 200, False), (12288, 1, 256, 140, True), (8192, 1, 256, 100, False)]
    dbs, jobs, exp = [], [], []
    for i, (n, d, z, B, masked) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=150, table=i)
        R = synth.random_bits(B, n, seed=151, table=i)
        db = _db(n, d, z, T)
        dbs.append(db)
        if masked:
            S = synth.mask_seeds(B, seed=152, table=i)
            dS = torch.from_numpy(np.ascontiguousarray(S)).cuda()
            jobs.append((db, B, to_dev(R), dev_out(B, d * z), dS))
            exp.append(oracle.read_batch_masked(T, n, d, z, R, S))
        else:
            jobs.append((db, B, to_dev(R), dev_out(B, d * z)))
            exp.append(oracle.read_batch(T, n, d, z, R))
    try:
        talekpir.read_multi_async(jobs)
        for job, e in zip(jobs, exp):
            assert np.array_equal(to_host(job[3]), e), job[0].n
        for job in jobs:
            job[3].zero_()
        g = talekpir.MultiGraph(jobs)
        g.launch()
        for job, e in zip(jobs, exp):
            assert np.array_equal(to_host(job[3]), e), job[0].n
        g.close()
    finally:
        for db in dbs:
            db.close()
    assert talekpir.device_status() == talekpir.OK
