"""Parity at the full sizes the benchmark times, through the C ABI:

- uneven batching: the 64 tables of synth.multi_table_shapes(64, seed=3)
  (16.6 GB; n = 2^U(10,17), d in {2,4,8}, 256 B..4 KiB messages, 16..512
  reads each) read by one replay of the captured many-table graph, then again
  after the autotuner has tuned every (row width, batch class) of them;
- the large table: n = 2^20 x 4 x 1 KiB (4 GiB), B = 1024 requests, on the
  automatic (tensor-core) kernel and the LOP3 kernel, the Four-Russians and
  plain kernels compared with them.

The oracle cannot redo a whole batch at this size, so every table is checked
on sampled rows (computed one by one by the oracle) and with GF(2) Freivalds
trials covering the whole batch: for a random subset S of the requests,
XOR_{b in S} Out[b] must equal the oracle's reply to XOR_{b in S} R[b] (the
reply is linear over XOR), and a wrong Out passes a trial with probability
at most 1/2.  The checks run in a spawn process pool on the host cores, each
worker rebuilding its table from the seeded host generator."""

import os

import numpy as np
import pytest

from gpu_helpers import dev_out, require_cuda, to_dev, to_host
from paper_2001_08250_gb300 import synth, talekpir
from workload_checks import check_generated_table, check_mapped_table, run_pool

pytestmark = pytest.mark.gpu

PLAIN, BATCHED, M4RM, TENSOR = 1, 2, 4, 5


def _sample_rows(B, k, seed):
    rng = np.random.default_rng(seed)
    rows = {0, B - 1}
    while len(rows) < min(B, k):
        rows.add(int(rng.integers(B)))
    return sorted(rows)


def test_uneven_batching_workload_as_benchmarked():
    torch = require_cuda()
    shapes = synth.multi_table_shapes(64, seed=3)
    jobs, Rs = [], []
    for i, (n, d, z, B) in enumerate(shapes):
        db = talekpir.DB(n, d, z)
        T = synth.table_bytes_torch(n, d, z, seed=3, table=i)
        db.load_async(T)
        torch.cuda.synchronize()
        del T
        R = synth.random_bits(B, n, seed=3, table=i)
        Rs.append(R)
        jobs.append((db, B, to_dev(R), dev_out(B, d * z)))

    def replay():
        g = talekpir.MultiGraph(jobs)
        for (_, _, _, dO) in jobs:
            dO.fill_(0xA5)
        g.launch()
        torch.cuda.synchronize()
        outs = [to_host(dO) for (_, _, _, dO) in jobs]
        g.close()
        return outs

    first = replay()
    # the benchmark's tuning: one trial per (row width, batch class), on the
    # class's smallest table
    seen = {}
    for (db, B, _, _) in jobs:
        key = (db.row_bytes, max(1, (B - 1).bit_length()))
        if key not in seen or db.n < seen[key][0].n:
            seen[key] = (db, B)
    for db, B in seen.values():
        db.autotune(B, reps=2)
    tuned = replay()
    talekpir.tune_clear()
    assert talekpir.device_status() == talekpir.OK
    tasks = [(i, n, d, z, 3, i, Rs[i], [first[i], tuned[i]], _sample_rows(B, 8, 100 + i), 20,
              200 + i) for i, (n, d, z, B) in enumerate(shapes)]
    for db, *_ in jobs:
        db.close()
    bad = [r for r in run_pool(check_generated_table, tasks) if r[1]]
    assert not bad, bad[:8]


def test_large_table_workload_tensor_and_lop3(tmp_path):
    """4 GiB table, B = 1024: 16 sampled rows and 20 Freivalds trials of the
    automatic kernel's replies (the tensor-core kernel at this batch); the LOP3
    and Four-Russians kernels' replies must equal them byte for byte (so the
    same checks hold for them), and the plain kernel's on four rows."""
    torch = require_cuda()
    n, d, z, B = 1 << 20, 4, 1024, 1024
    T = np.memmap(tmp_path / "table.bin", dtype=np.uint8, mode="w+", shape=(n, d * z))
    synth.table_bytes(n, d, z, seed=0, table=4, out=T)
    T.flush()
    R = synth.random_bits(B, n, seed=4)
    db = talekpir.DB(n, d, z)
    db.load(T)
    del T
    dR, dO = to_dev(R), dev_out(B, d * z)
    db.read_batch_async(dR, B, dO)
    Out = to_host(dO)
    for k in (BATCHED, M4RM):
        db.set_kernel(k)
        dO.fill_(0x5A)
        db.read_batch_async(dR, B, dO)
        assert np.array_equal(to_host(dO), Out), k
    db.set_kernel(PLAIN)
    dO1 = dev_out(4, d * z)
    db.read_batch_async(dR, 4, dO1)
    assert np.array_equal(to_host(dO1), Out[:4])
    torch.cuda.synchronize()
    db.close()
    assert talekpir.device_status() == talekpir.OK
    np.save(tmp_path / "R.npy", R)
    np.save(tmp_path / "Out.npy", Out)
    rows = _sample_rows(B, 16, 7)
    tasks = [(f"row {r}", str(tmp_path), n, d, z, [r], 0, 0) for r in rows]
    tasks += [(f"trial {t}", str(tmp_path), n, d, z, [], 1, 300 + t) for t in range(20)]
    bad = [r for r in run_pool(check_mapped_table, tasks) if r[1]]
    assert not bad, bad[:8]
