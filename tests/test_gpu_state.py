"""GPU parity of the server state: cuckoo writes (Section 5.3), interest
vectors (Section 7) and the continuous-batching serve loop, through the C ABI,
bit-exact against the oracle."""

import time

import numpy as np
import pytest

import oracle
from gpu_helpers import require_cuda
from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu


def _writes(count, n, z, seed):
    keys = synth.write_keys(count, seed=seed)
    b1, b2 = synth.bucket_pairs(keys, n)
    return b1, b2, synth.messages(count, z, seed=seed)


@pytest.mark.parametrize("n,d,z,cap,maxev,seed,batches", [
    (64, 4, 64, 240, 500, 11, [1, 7, 50, 100, 242]),   # high load, collection, evictions
    (32, 2, 16, 0, 30, 12, [64, 64]),                  # walks hit the bound: EFULL + rollback
    (256, 8, 48, 1500, 500, 13, [400, 400, 400]),      # d = 8, odd message size
    (1024, 4, 1024, 2048, 500, 0, [2048]),             # the plain-PIR workload's fill
])
def test_write_batches_match_oracle(n, d, z, cap, maxev, seed, batches):
    require_cuda()
    total = sum(batches)
    b1, b2, M = _writes(total, n, z, seed)
    oc = oracle.Cuckoo(n, d, z, cap, maxev, seed=seed)
    with talekpir.DB(n, d, z) as db:
        db.set_policy(cap, maxev, seed)
        i = 0
        nfull = 0
        for cnt in batches:
            st, ev = db.write_batch(b1[i:i + cnt], b2[i:i + cnt], M[i:i + cnt])
            for j in range(cnt):
                rc, oev = oc.insert(int(b1[i + j]), int(b2[i + j]), M[i + j])
                assert (int(st[j]), int(ev[j])) == (rc, oev), f"write {i + j}"
                nfull += rc == oracle.EFULL
            i += cnt
            assert np.array_equal(db.dump(), oc.table())
        assert db.epoch == total - nfull
    assert talekpir.device_status() == talekpir.OK


def test_tensor_reads_follow_writes_and_loads():
    """The tensor-core read uses a bit-transposed copy of the table, which
    every write (single writes with their moves in the launch, staged
    batches, the no-alloc write) and every bulk load must keep current: after
    each of them a forced tensor-core read of 100 requests equals the oracle's
    replies on the table at that point."""
    import ctypes
    torch = require_cuda()
    n, d, z, cap, seed = 3000, 2, 256, 5400, 71
    b1, b2, M = _writes(2600, n, z, seed)
    oc = oracle.Cuckoo(n, d, z, cap, 500, seed=seed)
    db = talekpir.DB(n, d, z)
    db.set_policy(cap, 500, seed)
    db.set_kernel(5)
    R = synth.random_bits(100, n, seed=seed + 1)

    def check(what):
        assert np.array_equal(db.read_batch(R), oracle.read_batch(oc.table(), n, d, z, R)), what

    check("empty table")            # builds the copy
    i = 0
    for count in (1, 1, 7, 300, 1, 900):   # parameter-passed moves and staged batches
        if count == 1:
            rc, _ = db.write(int(b1[i]), int(b2[i]), M[i])
            assert rc == oc.insert(int(b1[i]), int(b2[i]), M[i])[0]
        else:
            st, _ = db.write_batch(b1[i:i + count], b2[i:i + count], M[i:i + count])
            for j in range(count):
                assert st[j] == oc.insert(int(b1[i + j]), int(b2[i + j]), M[i + j])[0]
        i += count
        check(f"after {i} writes")
    dM = torch.from_numpy(M[i:i + 50]).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for j in range(50):
        ev = ctypes.c_uint32(0)
        rc = talekpir.lib().tpir_write_noalloc(db.h, int(b1[i + j]), int(b2[i + j]),
                                               dM[j].data_ptr(), ctypes.byref(ev), stream)
        assert rc == oc.insert(int(b1[i + j]), int(b2[i + j]), M[i + j])[0]
    torch.cuda.synchronize()
    check("after no-alloc writes")
    T2 = synth.table_bytes(n, d, z, seed=seed + 2)
    db.load(T2)
    assert np.array_equal(db.read_batch(R), oracle.read_batch(T2, n, d, z, R)), "after a load"
    db.close()
    assert talekpir.device_status() == talekpir.OK


def test_single_writes_and_rollback():
    require_cuda()
    n, d, z = 3, 1, 32
    oc = oracle.Cuckoo(n, d, z, 0, 20, seed=5)
    with talekpir.DB(n, d, z) as db:
        db.set_policy(0, 20, 5)
        for i, (a, b) in enumerate([(0, 1), (0, 1), (2, 2), (0, 1), (1, 2)]):
            msg = np.full(z, i + 1, dtype=np.uint8)
            before = db.dump()
            rc, ev = db.write(a, b, msg)
            assert (rc, ev) == oc.insert(a, b, msg)
            if rc == talekpir.EFULL:
                assert np.array_equal(db.dump(), before)
            assert np.array_equal(db.dump(), oc.table())
        with pytest.raises(talekpir.TpirError):
            db.write(3, 0, np.zeros(z, dtype=np.uint8))     # bucket out of range


def test_reads_see_writes_in_order():
    """A read submitted after a write sees it; one submitted before does not."""
    require_cuda()
    torch = require_cuda()
    n, d, z = 256, 4, 256
    b1, b2, M = _writes(300, n, z, 21)
    oc = oracle.Cuckoo(n, d, z, 0, 500, seed=21)
    R = synth.random_bits(8, n, seed=22)
    dR = torch.from_numpy(R.view(np.int64)).cuda()
    with talekpir.DB(n, d, z) as db:
        db.set_policy(0, 500, 21)
        outs = []
        for chunk in range(3):
            o = torch.empty((8, d * z), dtype=torch.uint8, device="cuda")
            db.read_batch_async(dR, 8, o)            # before this chunk's writes
            outs.append((o, oc.table()))
            sl = slice(chunk * 100, (chunk + 1) * 100)
            db.write_batch(b1[sl], b2[sl], M[sl])
            for j in range(sl.start, sl.stop):
                oc.insert(int(b1[j]), int(b2[j]), M[j])
        for o, T in outs:
            assert np.array_equal(o.cpu().numpy(), oracle.read_batch(T, n, d, z, R))
        assert np.array_equal(db.read_batch(R), oracle.read_batch(oc.table(), n, d, z, R))


@pytest.mark.parametrize("window,per_delta", [(1, 0), (4, 100), (2, 1)])
def test_interest_vector_matches_oracle(window, per_delta):
    require_cuda()
    m, k = 1 << 20, 4
    keys = synth.write_keys(1000, seed=31)
    P = synth.bloom_positions(keys, m, k)
    ob = oracle.Bloom(m, k, window, per_delta)
    with talekpir.DB(16, 1, 16) as db:
        db.bloom_create(m, k, window, per_delta)
        i = 0
        for cnt in (1, 3, 100, 250, 146):
            assert db.bloom_insert_batch(P[i:i + cnt]) == talekpir.OK
            for p in P[i:i + cnt]:
                ob.insert(p)
            i += cnt
            assert np.array_equal(db.bloom_get(), ob.get())
        vec = synth.random_bits(1, m, seed=32)[0]
        db.bloom_or_vector(vec)
        ob.or_vector(vec)
        assert np.array_equal(db.bloom_get(), ob.get())
        for p in P[i:]:
            assert db.bloom_insert(p) == talekpir.OK
            ob.insert(p)
        assert np.array_equal(db.bloom_get(), ob.get())
        bad = P[0].copy()
        bad[2] = m
        before = db.bloom_get()
        assert db.bloom_insert(bad) == talekpir.EINVAL
        assert np.array_equal(db.bloom_get(), before)


def _replay(shape, seed, writes, upto):
    """Oracle table of one serve table after its first `upto` successful writes
    (writes that failed are replayed too: they consume random draws)."""
    n, d, z = shape
    oc = oracle.Cuckoo(n, d, z, 0, 500, seed=seed)
    ok = 0
    for (b1, b2, msg) in writes:
        if ok == upto:
            break
        rc, _ = oc.insert(b1, b2, msg)
        ok += rc == 0
    return oc.table()


def test_serve_mix_each_result_same_alone_and_in_mix():
    """Reads and writes to three tables arrive interleaved; the server batches
    them across tables.  Every read's reply equals the oracle's answer on the
    table state its completion reports (epoch), i.e. the same as if the read
    had run alone at that point; the interest vectors match too."""
    require_cuda()
    shapes = [(512, 4, 256), (1024, 4, 1024), (300, 2, 64)]
    srv = talekpir.Server(hbm_budget_bytes=8 << 30, max_batch=32, max_inflight=3)
    tids, seeds = [], [41, 42, 43]
    for (n, d, z), sd in zip(shapes, seeds):
        tid = srv.add_table(n, d, z)
        db = srv.table(tid)
        db.set_policy(0, 500, sd)
        db.bloom_create(1 << 16, 3, window=2, writes_per_delta=40)
        tids.append(tid)
    total = 1500
    kind = synth.op_mix(total, 0.3, seed=44)
    which = (synth.stream(synth.stream_key(44, 1), total) % np.uint64(3)).astype(int)
    keys = synth.write_keys(total, seed=45)
    writes = {t: [] for t in tids}
    reads = {}
    outs = {}
    for i in range(total):
        t = int(which[i])
        n, d, z = shapes[t]
        if kind[i]:
            b1, b2 = synth.bucket_pairs(keys[i:i + 1], n)
            msg = synth.messages(1, z, seed=1000 + i)[0]
            pos = synth.bloom_positions(keys[i:i + 1], 1 << 16, 3)[0]
            writes[t].append((int(b1[0]), int(b2[0]), msg, pos))
            while srv.submit_write(t, int(b1[0]), int(b2[0]), msg, i, pos) == talekpir.EAGAIN:
                time.sleep(0.001)
        else:
            q = synth.random_bits(1, n, seed=2000 + i)[0]
            outs[i] = np.empty(d * z, dtype=np.uint8)
            reads[i] = (t, q)
            while srv.submit_read(t, q, outs[i], i) == talekpir.EAGAIN:
                time.sleep(0.001)
        if i % 97 == 0:
            time.sleep(0.002)   # let launches form while more ops arrive
    srv.drain()
    comps = srv.poll(100000)
    assert len(comps) == total
    assert all(c.status == 0 for c in comps if c.kind == 0)
    st = srv.stats()
    assert st.reads_done == len(reads) and st.launches >= 2
    cache = {}
    for c in comps:
        if c.kind != 0:
            continue
        t, q = reads[c.tag]
        key = (t, c.epoch)
        if key not in cache:
            cache[key] = _replay(shapes[t], seeds[t], [w[:3] for w in writes[t]], c.epoch)
        n, d, z = shapes[t]
        assert np.array_equal(outs[c.tag], oracle.read(cache[key], n, d, z, q)), c.tag
    # interest vectors: successful writes' positions in arrival order
    for t in tids:
        ob = oracle.Bloom(1 << 16, 3, 2, 40)
        oc = oracle.Cuckoo(*shapes[t], 0, 500, seed=seeds[t])
        for (b1, b2, msg, pos) in writes[t]:
            if oc.insert(b1, b2, msg)[0] == 0:
                ob.insert(pos)
        assert np.array_equal(srv.table(t).bloom_get(), ob.get())
    srv.close()


def test_serve_bursts_reach_the_tensor_core_kernel():
    """Reads arrive in bursts of 300 per table with writes between them.  With
    a batching window (tick_us) a table's burst is read in launches of up to
    max_batch = 256 requests, which take the tensor-core kernel (48 or more
    requests on rows of 256 bytes or more); the rest of each burst takes the
    register-tiled kernel.  Every read equals the oracle's answer on the table
    state its completion reports, and the server's launch counts show the
    tensor-core kernel ran inside the serve loop."""
    require_cuda()
    shapes = [(4096, 4, 1024), (3000, 2, 256)]
    seeds = [61, 62]
    srv = talekpir.Server(hbm_budget_bytes=8 << 30, max_batch=256, max_inflight=2,
                          tick_us=20000)
    for (n, d, z), sd in zip(shapes, seeds):
        tid = srv.add_table(n, d, z)
        srv.table(tid).set_policy(0, 500, sd)
    writes = {0: [], 1: []}
    reads, outs = {}, {}
    tag = 0
    for burst in range(3):
        for t, (n, d, z) in enumerate(shapes):
            keys = synth.write_keys(5, seed=700 + 10 * burst + t)
            b1, b2 = synth.bucket_pairs(keys, n)
            msgs = synth.messages(5, z, seed=800 + 10 * burst + t)
            for j in range(5):
                writes[t].append((int(b1[j]), int(b2[j]), msgs[j]))
                assert srv.submit_write(t, int(b1[j]), int(b2[j]), msgs[j], tag) == talekpir.OK
                tag += 1
            R = synth.random_bits(300, n, seed=900 + 10 * burst + t)
            for q in R:
                outs[tag] = np.empty(d * z, dtype=np.uint8)
                reads[tag] = (t, q)
                assert srv.submit_read(t, q, outs[tag], tag) == talekpir.OK
                tag += 1
        srv.drain()
    comps = srv.poll(100000)
    assert len(comps) == tag
    assert all(c.status == 0 for c in comps)
    st = srv.stats()
    assert st.reads_done == len(reads)
    assert st.kernel_launches[5] >= 2, list(st.kernel_launches)
    assert st.mean_batch >= 48
    cache = {}
    for c in comps:
        if c.kind != 0:
            continue
        t, q = reads[c.tag]
        key = (t, c.epoch)
        if key not in cache:
            cache[key] = _replay(shapes[t], seeds[t], writes[t], c.epoch)
        n, d, z = shapes[t]
        assert np.array_equal(outs[c.tag], oracle.read(cache[key], n, d, z, q)), c.tag
    srv.close()


def test_serve_budget_and_backpressure():
    require_cuda()
    srv = talekpir.Server(hbm_budget_bytes=1 << 30, max_batch=8, max_inflight=2, queue_capacity=4)
    srv.add_table(1 << 15, 4, 1024)                      # 128 MiB
    with pytest.raises(talekpir.TpirError) as e:
        srv.add_table(1 << 18, 4, 1024)                  # 1 GiB: over the budget
    assert e.value.status == talekpir.ENOMEM
    q = synth.random_bits(1, 1 << 15, seed=1)[0]
    outs = [np.empty(4096, dtype=np.uint8) for _ in range(64)]
    rcs = [srv.submit_read(0, q, outs[i], i) for i in range(64)]
    assert talekpir.EAGAIN in rcs and talekpir.OK in rcs
    srv.drain()
    st = srv.stats()
    assert st.rejected == rcs.count(talekpir.EAGAIN)
    assert st.reads_done == rcs.count(talekpir.OK)
    srv.close()


def test_bounded_wait_gives_up_and_context_survives():
    """Failure detection without a GPU fault: a kernel waits on a barrier that
    nothing arrives at; the bounded wait gives up after 20 ms, the status word
    reports TPIR_ETIMEDOUT, and the context keeps serving exact reads."""
    require_cuda()
    t0 = time.perf_counter()
    assert talekpir.lib().tpir_selftest_wait_timeout(20000) == talekpir.ETIMEDOUT
    assert time.perf_counter() - t0 < 5.0
    assert talekpir.device_status() == talekpir.OK          # the word was cleared
    n, d, z = 300, 2, 64
    T = synth.table_bytes(n, d, z, seed=70)
    R = synth.random_bits(9, n, seed=71)
    with talekpir.DB(n, d, z) as db:
        db.load(T)
        assert np.array_equal(db.read_batch(R), oracle.read_batch(T, n, d, z, R))
    assert talekpir.lib().tpir_selftest_wait_timeout(0) == talekpir.EINVAL


def test_real_read_with_second_bucket_retry():
    """A client's RealRead (Section 5.4): messages written through the cuckoo
    path sit in one of their two buckets (evictions may move them), so a read
    asks for the first bucket with three XOR shares (Section 2), looks for the
    message's tag among the d slots of the reconstructed bucket, and only if
    it is absent asks for the second bucket.  Every message is found, some
    only on the retry; each reconstructed bucket equals the oracle table's."""
    require_cuda()
    n, d, z, count = 256, 4, 64, 700
    keys = synth.write_keys(count, seed=41)
    b1, b2 = synth.bucket_pairs(keys, n)
    msgs = synth.messages(count, z, seed=41)
    msgs[:, :8] = np.arange(1, count + 1, dtype=np.uint64).view(np.uint8).reshape(count, 8)  # tag
    db = talekpir.DB(n, d, z)
    db.set_policy(0, 500, 41)
    oc = oracle.Cuckoo(n, d, z, 0, 500, seed=41)
    live = []
    for i in range(count):
        rc, _ = db.write(int(b1[i]), int(b2[i]), msgs[i])
        assert rc == oc.insert(int(b1[i]), int(b2[i]), msgs[i])[0]
        if rc == talekpir.OK:
            live.append(i)
    T = oc.table()
    want = np.array(live[::7])
    retries = 0

    def read_bucket(targets):
        sh = synth.xor_shares(n, targets, 3, seed=42 + len(targets))
        got = db.read_batch(sh.reshape(len(targets) * 3, -1)).reshape(len(targets), 3, -1)
        return got[:, 0] ^ got[:, 1] ^ got[:, 2]

    first = read_bucket(b1[want].astype(np.int64))
    assert np.array_equal(first, T[b1[want]])
    missing = []
    for j, i in enumerate(want):
        slots = first[j].reshape(d, z)
        if not any(np.array_equal(s, msgs[i]) for s in slots):
            missing.append(i)
    retries = len(missing)
    if missing:
        second = read_bucket(b2[np.array(missing)].astype(np.int64))
        assert np.array_equal(second, T[b2[np.array(missing)]])
        for j, i in enumerate(missing):
            slots = second[j].reshape(d, z)
            assert any(np.array_equal(s, msgs[i]) for s in slots), i
    assert retries > 0                      # some messages live in their second bucket
    assert retries < len(want)
    db.close()
    assert talekpir.device_status() == talekpir.OK
