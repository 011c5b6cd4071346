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
