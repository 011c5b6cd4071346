"""CPU tests of the row-sharded read path (the scale-out Section 9.4 proposes):
the shard plan, argument checks of tpir_db_create_shard, and the XOR exchange
across torch.distributed ranks on the gloo backend (world sizes 2 and 3).

The server answer is linear over XOR in the buckets, so the XOR of the
partial answers over a partition of the rows is the whole answer; the
exchange test computes each rank's partial with the oracle on that rank's
rows and checks the exchanged reply against the oracle's full answer."""

import os
import socket

import numpy as np
import pytest

import oracle
from paper_2001_08250_gb300 import synth, talekpir


@pytest.mark.parametrize("n_total,parts", [(1, 1), (64, 1), (65, 2), (100, 4), (32768, 3),
                                           (32768, 8), (1 << 20, 7), (129, 3), (5000, 64)])
def test_shard_plan_partitions_whole_words(n_total, parts):
    plan = talekpir.shard_plan(n_total, parts)
    assert len(plan) == parts
    pos = 0
    for begin, rows in plan:
        assert begin % 64 == 0
        if rows:
            assert begin == pos
            pos += rows
    assert pos == n_total
    nonempty = [r for _, r in plan if r]
    words = (n_total + 63) // 64
    assert len(nonempty) == min(parts, words)
    # balanced to one request word, except the ragged last word
    full = [r for b, r in plan if r and b + r < n_total]
    if full:
        assert max(full) - min(full) <= 64


def test_create_shard_rejects_bad_ranges():
    L = talekpir.lib()
    for args in [(0, 0, 1), (100, 10, 5), (100, 64, 37), (100, 128, 1), (100, 0, 0)]:
        assert L.tpir_db_create_shard(args[0], args[1], args[2], 4, 1024) is None
        assert L.tpir_last_error() == talekpir.EINVAL
    assert L.tpir_shard_plan(100, 0, 0, None, None) == talekpir.EINVAL


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _exchange_rank(rank, world, port, n, d, z, B, result_dir):
    import torch
    import torch.distributed as dist

    from paper_2001_08250_gb300 import shard

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        T = synth.table_bytes(n, d, z, seed=90)
        R = synth.random_bits(B, n, seed=91)
        begin, rows = talekpir.shard_plan(n, world)[rank]
        if rows:
            w0 = begin // 64
            Rs = np.ascontiguousarray(R[:, w0:w0 + (rows + 63) // 64])
            part = oracle.read_batch(T[begin:begin + rows], rows, d, z, Rs)
        else:
            part = np.zeros((B, d * z), dtype=np.uint8)

        def np_combine(parts, out):
            acc = np.bitwise_xor.reduce(np.stack([p.numpy() for p in parts]), axis=0)
            out.copy_(torch.from_numpy(acc))

        got = shard.xor_exchange(torch.from_numpy(part), combine=np_combine).numpy()
        ok = np.array_equal(got, oracle.read_batch(T, n, d, z, R))
        # the device combine refuses CPU tensors instead of falling back
        try:
            shard.xor_exchange(torch.from_numpy(part))
            refused = False
        except RuntimeError:
            refused = True
        with open(os.path.join(result_dir, f"rank{rank}"), "w") as f:
            f.write(f"{int(ok)} {int(refused)}")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 1000), (3, 130), (2, 64)])
def test_xor_exchange_over_gloo_ranks(world, n, tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    d, z, B = 2, 64, 5
    mp.spawn(_exchange_rank, args=(world, _free_port(), n, d, z, B, str(tmp_path)),
             nprocs=world, join=True)
    for r in range(world):
        assert (tmp_path / f"rank{r}").read_text() == "1 1", r
