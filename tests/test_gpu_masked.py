"""GPU parity of serialized-PIR masked reads (Section 6, steps 5-9) against
the oracle, through the C ABI.

Every masked reply must equal the oracle's R_b XOR PRNG(p_b) byte for byte,
for every read kernel, on small and ragged shapes (rows that end inside a
64-byte keystream block), at paper scale on sampled rows in the launch
configuration the benchmark times, and in many-table launches; the leader's
XOR and the client's mask removal recover the target bucket."""

import numpy as np
import pytest

import oracle
from gpu_helpers import dev_out, require_cuda, to_dev, to_host
from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu

PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR = 1, 2, 3, 4, 5

EDGE = [
    (1, 1, 16, 1), (63, 1, 16, 3), (64, 2, 48, 9), (65, 4, 16, 31), (200, 8, 32, 33),
    (333, 2, 256, 64), (1000, 1, 4096, 17), (1024, 4, 1024, 257), (777, 3, 80, 12),
    (130, 8, 4096, 8), (2049, 1, 64, 100), (1500, 2, 512, 520),
]


def _db(n, d, z, T):
    db = talekpir.DB(n, d, z)
    db.load(T)
    return db


def _seeds_dev(S):
    torch = require_cuda()
    return torch.from_numpy(np.ascontiguousarray(S)).cuda()


@pytest.mark.parametrize("n,d,z,B", EDGE)
@pytest.mark.parametrize("kernel", [PLAIN, BATCHED, PLAIN_REG, M4RM, TENSOR])
def test_masked_edge_shapes_bit_exact(n, d, z, B, kernel):
    require_cuda()
    T = synth.table_bytes(n, d, z, seed=61, table=n * 5 + d)
    R = synth.random_bits(B, n, seed=62, table=n)
    S = synth.mask_seeds(B, seed=63, table=n)
    exp = oracle.read_batch_masked(T, n, d, z, R, S)
    with _db(n, d, z, T) as db:
        db.set_kernel(kernel)
        assert np.array_equal(db.read_batch_masked(R, S), exp)
        dR, dS, dO = to_dev(R), _seeds_dev(S), dev_out(B, d * z)
        db.read_batch_masked_async(dR, B, dS, dO)
        assert np.array_equal(to_host(dO), exp)
        # the unmasked read of the same requests is untouched by the masks
        assert np.array_equal(db.read_batch(R), oracle.read_batch(T, n, d, z, R))
    assert talekpir.device_status() == talekpir.OK


def test_masked_paper_scale_sampled():
    """n = 32768, d = 4, 1 KiB messages (128 MiB), 256 masked Bernoulli(0.5)
    requests through the device-buffer entry point (the automatic kernel
    choice, as benchmarked); sampled rows against the oracle, and the forced
    kernels agree with it on the whole batch."""
    require_cuda()
    n, d, z, B = 32768, 4, 1024, 256
    T = synth.table_bytes(n, d, z, seed=0)
    R = synth.random_bits(B, n, seed=64)
    S = synth.mask_seeds(B, seed=64)
    rows = [0, 1, 127, 255]
    with _db(n, d, z, T) as db:
        dR, dS, dO = to_dev(R), _seeds_dev(S), dev_out(B, d * z)
        db.read_batch_masked_async(dR, B, dS, dO)
        Out = to_host(dO)
        exp = oracle.read_batch_masked(T, n, d, z, R[rows], S[rows])
        assert np.array_equal(Out[rows], exp)
        for k in (BATCHED, M4RM, TENSOR):
            db.set_kernel(k)
            dO2 = dev_out(B, d * z)
            db.read_batch_masked_async(dR, B, dS, dO2)
            assert np.array_equal(to_host(dO2), Out)
        db.set_kernel(PLAIN)
        dO1 = dev_out(4, d * z)
        db.read_batch_masked_async(dR[:4], 4, dS[:4], dO1)
        assert np.array_equal(to_host(dO1), Out[:4])
    assert talekpir.device_status() == talekpir.OK


@pytest.mark.parametrize("rows,nbytes", [(1, 16), (3, 48), (5, 64), (7, 80), (16, 4096),
                                         (2, 65536 + 16), (300, 1024)])
def test_mask_generate_matches_oracle(rows, nbytes):
    torch = require_cuda()
    S = synth.mask_seeds(rows, seed=65, table=nbytes)
    out = torch.empty((rows, nbytes), dtype=torch.uint8, device="cuda")
    talekpir.mask_generate(_seeds_dev(S), rows, nbytes, out)
    got = to_host(out)
    for b in range(rows):
        assert np.array_equal(got[b], oracle.mask(S[b], nbytes)), b


@pytest.mark.parametrize("count,nbytes", [(1, 16), (3, 4096), (64, 1 << 20)])
def test_xor_combine(count, nbytes):
    torch = require_cuda()
    bufs = [torch.from_numpy(synth.messages(1, nbytes, seed=66, table=k)[0]).cuda()
            for k in range(count)]
    ref = np.bitwise_xor.reduce(np.stack([to_host(b) for b in bufs]), axis=0)
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    talekpir.xor_combine(bufs, nbytes, dst)
    assert np.array_equal(to_host(dst), ref)
    # in place: the destination is the first source
    talekpir.xor_combine(bufs, nbytes, bufs[0])
    assert np.array_equal(to_host(bufs[0]), ref)


def test_serialized_pir_three_servers_end_to_end():
    """Section 6 with l = 3 servers on the plain-PIR shape (n = 1024, d = 4,
    1 KiB): each server answers its XOR share masked by its own seeds; the
    leader combines the three masked replies on the device; the client's
    masks, generated on the device and combined, remove the masks and leave
    exactly the target buckets."""
    torch = require_cuda()
    n, d, z, l, Q = 1024, 4, 1024, 3, 64
    T = synth.table_bytes(n, d, z, seed=67)
    tg = synth.targets(Q, n, seed=67)
    shares = synth.xor_shares(n, tg, l, seed=67)
    seeds = [synth.mask_seeds(Q, seed=67, server=i) for i in range(l)]
    servers = [_db(n, d, z, T) for _ in range(l)]   # each server holds its replica
    replies = []
    for i, db in enumerate(servers):
        dO = dev_out(Q, d * z)
        db.read_batch_masked_async(to_dev(np.ascontiguousarray(shares[:, i, :])), Q,
                                   _seeds_dev(seeds[i]), dO)
        replies.append(dO)
        # a single server's reply is masked: it is not the plain answer
        assert not np.array_equal(to_host(dO),
                                  oracle.read_batch(T, n, d, z, shares[:, i, :]))
    leader = dev_out(Q, d * z)
    talekpir.xor_combine(replies, Q * d * z, leader)
    masks = []
    for i in range(l):
        m = dev_out(Q, d * z)
        talekpir.mask_generate(_seeds_dev(seeds[i]), Q, d * z, m)
        masks.append(m)
    client = dev_out(Q, d * z)
    talekpir.xor_combine([leader] + masks, Q * d * z, client)
    torch.cuda.synchronize()
    assert np.array_equal(to_host(client), T[tg])
    for db in servers:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_masked_jobs_in_many_table_launches_and_graph():
    """Masked and plain jobs mixed in one call: small batches (register-tiled
    launch), large batches on 256- and 512-request Four-Russians tiles; the
    captured graph replays give the same replies."""
    torch = require_cuda()
    shapes = [(1100, 2, 256, 16, True), (3000, 4, 1024, 40, False), (513, 8, 4096, 7, True),
              (2048, 2, 256, 300, True), (700, 8, 256, 200, True), (4096, 4, 1024, 256, False),
              (97, 1, 16, 1, True), (2049, 2, 512, 333, False)]
    dbs, jobs, exp = [], [], []
    for i, (n, d, z, B, masked) in enumerate(shapes):
        T = synth.table_bytes(n, d, z, seed=70, table=i)
        R = synth.random_bits(B, n, seed=71, table=i)
        db = _db(n, d, z, T)
        dbs.append(db)
        if masked:
            S = synth.mask_seeds(B, seed=72, table=i)
            jobs.append((db, B, to_dev(R), dev_out(B, d * z), _seeds_dev(S)))
            exp.append(oracle.read_batch_masked(T, n, d, z, R, S))
        else:
            jobs.append((db, B, to_dev(R), dev_out(B, d * z), None))
            exp.append(oracle.read_batch(T, n, d, z, R))
    talekpir.read_multi_async(jobs)
    for j, e in zip(jobs, exp):
        assert np.array_equal(to_host(j[3]), e)
    g = talekpir.MultiGraph(jobs)
    for rep in range(2):
        for j in jobs:
            j[3].fill_(0xA5)
        g.launch()
        torch.cuda.synchronize()
        for j, e in zip(jobs, exp):
            assert np.array_equal(to_host(j[3]), e), rep
    g.close()
    for db in dbs:
        db.close()
    assert talekpir.device_status() == talekpir.OK


def test_masked_read_argument_errors():
    torch = require_cuda()
    n, d, z, B = 100, 2, 64, 4
    with _db(n, d, z, synth.table_bytes(n, d, z, seed=73)) as db:
        R = to_dev(synth.random_bits(B, n, seed=73))
        S = torch.zeros(B * 32 + 16, dtype=torch.uint8, device="cuda")
        O = dev_out(B, d * z)
        L = talekpir.lib()
        # seeds missing, or not 16-byte aligned
        assert L.tpir_read_batch_masked_async(db.h, R.data_ptr(), B, None, O.data_ptr(), None) \
            == talekpir.EINVAL
        assert L.tpir_read_batch_masked_async(db.h, R.data_ptr(), B, S.data_ptr() + 8,
                                              O.data_ptr(), None) == talekpir.EINVAL
        # mask lengths must be whole 16-byte words; combine needs 1..64 sources
        assert L.tpir_mask_generate(S.data_ptr(), 1, 40, O.data_ptr(), None) == talekpir.EINVAL
        assert L.tpir_xor_combine(None, 0, 16, O.data_ptr(), None) == talekpir.EINVAL
    assert talekpir.device_status() == talekpir.OK
