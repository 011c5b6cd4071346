"""GPU test of tpir_write_noalloc, the cuckoo write for callers that cannot
allocate device memory (a serving thread that cannot stall on cudaMalloc, a
process whose device memory belongs to another allocator).  It must leave the
table exactly as tpir_write does, call after call, through the C ABI.

Collected last on purpose: if it fails, a run stopped at the first failure
has already run every other test.  It also passes alone in a fresh process
(its first call on the device looks up the scratch array's address)."""

import ctypes

import numpy as np
import pytest

from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu


def _noalloc(db, b1, b2, d_msg, stream=0):
    ev = ctypes.c_uint32(0)
    rc = talekpir.lib().tpir_write_noalloc(db.h, int(b1), int(b2), d_msg.data_ptr(),
                                           ctypes.byref(ev), stream)
    return rc, ev.value


@pytest.mark.parametrize("n,d,z,cap,seed,count", [
    (64, 4, 1024, 240, 7, 300),     # high load: eviction chains and collection
    (16, 2, 65536, 0, 8, 40),       # the largest slot the scratch holds
])
def test_noalloc_write_matches_tpir_write(n, d, z, cap, seed, count):
    import torch
    assert torch.cuda.is_available()
    keys = synth.write_keys(count, seed=seed)
    b1, b2 = synth.bucket_pairs(keys, n)
    M = synth.messages(count, z, seed=seed)
    dM = torch.from_numpy(M).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    ref = talekpir.DB(n, d, z)
    new = talekpir.DB(n, d, z)
    for db in (ref, new):
        db.set_policy(cap, 500, seed)
    evictions = 0
    for i in range(count):
        rc_ref, ev_ref = ref.write(int(b1[i]), int(b2[i]), M[i])
        rc_new, ev_new = _noalloc(new, b1[i], b2[i], dM[i], stream)
        assert (rc_new, ev_new) == (rc_ref, ev_ref), f"write {i}"
        evictions += ev_ref
        if i < 4 or i % 37 == 0 or i == count - 1:
            torch.cuda.synchronize()
            assert np.array_equal(new.dump(), ref.dump()), f"table after write {i}"
    assert new.epoch == ref.epoch
    # reads see the same table
    R = synth.random_bits(8, n, seed=seed + 1)
    assert np.array_equal(new.read_batch(R), ref.read_batch(R))
    if cap:
        assert evictions > 0
    ref.close()
    new.close()
    assert talekpir.device_status() == talekpir.OK


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    assert torch.cuda.is_available()
    big = talekpir.DB(4, 1, 65536 + 16)
    msg = torch.zeros(65536 + 16, dtype=torch.uint8, device="cuda")
    rc, _ = _noalloc(big, 0, 1, msg)
    assert rc == talekpir.EINVAL
    assert not big.dump().any() and big.epoch == 0
    big.close()
    db = talekpir.DB(4, 1, 64)
    db.set_policy(0, 501, 0)               # walks longer than the scratch path accepts
    rc, _ = _noalloc(db, 0, 1, torch.zeros(64, dtype=torch.uint8, device="cuda"))
    assert rc == talekpir.EINVAL and db.epoch == 0
    db.close()


def _seed_with_even_first_draw() -> int:
    """A cuckoo seed whose first random draw has bit 0 clear (the walk then
    starts at the new item's first bucket)."""
    for s in range(1000):
        if synth.splitmix64_sequence(s, 1)[0] & 1 == 0:
            return s
    raise AssertionError("no seed found")


def test_noalloc_move_cycle_goes_through_the_scratch_slot():
    """A hand-traced insertion whose slot moves form a cycle, so that the
    write must park a slot in the file-scope scratch array.  n = 4 buckets of
    one slot each, 64 KiB messages (the largest the scratch holds).  P sits in
    bucket 0 (candidates 0, 1), Q in bucket 1 (1, 0), R in bucket 2 (2, 3).
    X (candidates 0, 2) finds both buckets full; with an even first draw the
    walk starts at bucket 0: X -> 0 evicts P, P -> 1 evicts Q, Q -> 0 evicts X,
    X -> 2 evicts R, R -> 3 (free): 4 evictions.  P and Q swap slots 0 and 1,
    which copies between slots can only do through a third slot: the scratch.
    Final layout: Q, P, X, R."""
    import torch
    n, d, z = 4, 1, 65536
    seed = _seed_with_even_first_draw()
    M = synth.messages(4, z, seed=21)
    P, Q, R, X = M
    dM = torch.from_numpy(M).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    pairs = [(0, 1), (1, 0), (2, 3), (0, 2)]
    new = talekpir.DB(n, d, z)
    ref = talekpir.DB(n, d, z)
    for db in (new, ref):
        db.set_policy(0, 500, seed)
    for _ in range(2):   # twice in a row: the scratch keeps the previous call's bytes
        for i, (b1, b2) in enumerate(pairs):
            rc, ev = _noalloc(new, b1, b2, dM[i], stream)
            rc_ref, ev_ref = ref.write(b1, b2, M[i])
            assert (rc, ev) == (rc_ref, ev_ref) == (0, 4 if i == 3 else 0), (i, rc, ev)
        torch.cuda.synchronize()
        expected = np.stack([Q, P, X, R])
        assert np.array_equal(new.dump().reshape(n, z), expected)
        assert np.array_equal(ref.dump().reshape(n, z), expected)
        for db in (new, ref):   # the same walk again on an emptied table
            db.load(np.zeros(n * z, dtype=np.uint8))
            db.set_policy(0, 500, seed)
    new.close()
    ref.close()
    assert talekpir.device_status() == talekpir.OK


def test_noalloc_writes_on_two_streams_stay_in_order():
    """Writes to one table alternate between two streams; each runs after the
    previous one whatever stream that used, so the table, and a read of it,
    equal those of the same writes through tpir_write."""
    import torch
    n, d, z, cap, count = 64, 4, 1024, 240, 200
    keys = synth.write_keys(count, seed=31)
    b1, b2 = synth.bucket_pairs(keys, n)
    M = synth.messages(count, z, seed=31)
    dM = torch.from_numpy(M).cuda()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ref = talekpir.DB(n, d, z)
    new = talekpir.DB(n, d, z)
    for db in (ref, new):
        db.set_policy(cap, 500, 31)
    for i in range(count):
        rc_ref, ev_ref = ref.write(int(b1[i]), int(b2[i]), M[i])
        rc, ev = _noalloc(new, b1[i], b2[i], dM[i], streams[i & 1].cuda_stream)
        assert (rc, ev) == (rc_ref, ev_ref), f"write {i}"
    R = synth.random_bits(16, n, seed=32)
    assert np.array_equal(new.read_batch(R), ref.read_batch(R))
    torch.cuda.synchronize()
    assert np.array_equal(new.dump(), ref.dump())
    ref.close()
    new.close()
    assert talekpir.device_status() == talekpir.OK
