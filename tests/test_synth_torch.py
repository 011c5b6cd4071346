"""The torch form of the input generator (used to fill multi-gigabyte tables
on the device) gives exactly the bytes of the numpy form, on the CPU: random
keys, offsets past 2^32 words, and whole tables."""

import numpy as np

from paper_2001_08250_gb300 import synth


def test_stream_torch_equals_stream():
    for i, start in enumerate([0, 1, 12345, (1 << 32) - 3, (1 << 40) + 7]):
        key = synth.stream_key(101, i)
        a = synth.stream(key, 4099, start)
        b = synth.stream_torch(key, 4099, start, device="cpu").numpy().view(np.uint64)
        assert np.array_equal(a, b)


def test_table_bytes_torch_equals_table_bytes():
    for (n, d, z, table) in [(1, 1, 16, 0), (100, 2, 256, 7), (1000, 4, 1024, 3)]:
        a = synth.table_bytes(n, d, z, seed=3, table=table)
        b = synth.table_bytes_torch(n, d, z, seed=3, table=table, device="cpu").numpy()
        assert np.array_equal(a, b)
