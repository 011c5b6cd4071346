"""GPU parity of row-sharded reads (the scale-out Section 9.4 proposes),
through the C ABI, with the shards of one table emulated on one GPU in one
process: every shard reads the same full-length request rows, and the XOR of
the shards' partial replies (the exchange's combine kernel) must equal the
oracle's answer for the whole table, byte for byte, for every read kernel."""

import numpy as np
import pytest

import oracle
from gpu_helpers import check_rows, dev_out, require_cuda, to_dev, to_host
from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu


def _shards(n, d, z, T, parts):
    dbs = []
    for begin, rows in talekpir.shard_plan(n, parts):
        if not rows:
            continue
        db = talekpir.DB(rows, d, z, shard=(n, begin))
        db.load(T[begin:begin + rows])
        dbs.append(db)
    return dbs


def _combine(parts, B, row):
    out = dev_out(B, row)
    talekpir.xor_combine(parts, B * row, out)
    return to_host(out)


@pytest.mark.parametrize("n,d,z,B", [(4097, 2, 256, 40), (1000, 4, 1024, 260), (130, 1, 16, 3),
                                     (2049, 8, 512, 180)])
@pytest.mark.parametrize("parts", [1, 2, 3, 5])
@pytest.mark.parametrize("kernel", [0, 1, 2, 4, 5])
def test_sharded_read_bit_exact(n, d, z, B, parts, kernel):
    require_cuda()
    T = synth.table_bytes(n, d, z, seed=92, table=n)
    R = synth.random_bits(B, n, seed=93, table=n)
    exp = oracle.read_batch(T, n, d, z, R)
    dR = to_dev(R)
    dbs = _shards(n, d, z, T, parts)
    partials = []
    for db in dbs:
        db.set_kernel(kernel)
        dO = dev_out(B, d * z)
        db.read_batch_async(dR, B, dO)
        partials.append(dO)
    assert np.array_equal(_combine(partials, B, d * z), exp)
    # the host-buffer entry point reads full-length rows as well
    host = [db.read_batch(R) for db in dbs]
    assert np.array_equal(np.bitwise_xor.reduce(np.stack(host), axis=0), exp)
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_sharded_masked_and_many_table_launch():
    """Shards of two tables in one many-table call; the first table's reply
    is masked on its first shard only, so the combined reply is the masked
    reply of the whole table."""
    require_cuda()
    tabs = [(3000, 4, 1024, 200), (777, 2, 256, 33)]
    jobs, plans, exps = [], [], []
    for t, (n, d, z, B) in enumerate(tabs):
        T = synth.table_bytes(n, d, z, seed=94, table=t)
        R = synth.random_bits(B, n, seed=95, table=t)
        dR = to_dev(R)
        S = synth.mask_seeds(B, seed=96, table=t) if t == 0 else None
        dS = to_dev(S) if S is not None else None
        dbs = _shards(n, d, z, T, 3)
        outs = []
        for i, db in enumerate(dbs):
            dO = dev_out(B, d * z)
            jobs.append((db, B, dR, dO, dS if i == 0 else None))
            outs.append(dO)
        plans.append((dbs, outs, B, d * z))
        exps.append(oracle.read_batch_masked(T, n, d, z, R, S) if S is not None
                    else oracle.read_batch(T, n, d, z, R))
    talekpir.read_multi_async(jobs)
    for (dbs, outs, B, row), e in zip(plans, exps):
        assert np.array_equal(_combine(outs, B, row), e)
        for db in dbs:
            db.close()
    assert talekpir.device_status() == talekpir.OK


def test_paper_scale_four_shards_sampled():
    """n = 32768, d = 4, 1 KiB messages (128 MiB) in four row shards, 256
    Bernoulli(0.5) requests (the automatic kernel choice): the combined
    replies equal the unsharded read and, on sampled rows, the oracle."""
    require_cuda()
    n, d, z, B = 32768, 4, 1024, 256
    T = synth.table_bytes(n, d, z, seed=0)
    R = synth.random_bits(B, n, seed=97)
    dR = to_dev(R)
    dbs = _shards(n, d, z, T, 4)
    parts = []
    for db in dbs:
        dO = dev_out(B, d * z)
        db.read_batch_async(dR, B, dO)
        parts.append(dO)
    got = _combine(parts, B, d * z)
    check_rows(T, n, d, z, R, got, [0, 100, 255])
    with talekpir.DB(n, d, z) as full:
        full.load(T)
        assert np.array_equal(got, full.read_batch(R))
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_shards_refuse_cuckoo_writes():
    torch = require_cuda()
    n, d, z = 256, 2, 64
    db = talekpir.DB(128, d, z, shard=(n, 128))
    msg = synth.messages(1, z, seed=98)[0]
    with pytest.raises(talekpir.TpirError):
        db.write(1, 2, msg)
    dmsg = torch.from_numpy(msg).cuda()
    import ctypes
    e = ctypes.c_uint32(0)
    assert talekpir.lib().tpir_write_noalloc(db.h, 1, 2, dmsg.data_ptr(), ctypes.byref(e), None) \
        == talekpir.EINVAL
    nt, rb = ctypes.c_uint64(), ctypes.c_uint64()
    assert talekpir.lib().tpir_db_shard_info(db.h, ctypes.byref(nt), ctypes.byref(rb)) == 0
    assert (nt.value, rb.value) == (n, 128)
    db.close()
