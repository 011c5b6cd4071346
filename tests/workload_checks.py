"""Oracle checks of full-size workloads, run in a process pool (test harness
only).  The pool is started with the "spawn" method: the parent process has a
CUDA context, and a worker forked from it could hang.  Each task rebuilds its
inputs from the seeded generators (or maps the parent's table file), so no
input reaches the oracle through the GPU."""

from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _rows_and_freivalds(T, n, d, z, R, Out, rows, trials, seed):
    import oracle
    for b in rows:
        exp = oracle.read(T, n, d, z, R[b])
        if not np.array_equal(Out[b], exp):
            return f"row {b} differs"
    rng = np.random.default_rng(seed)
    B = R.shape[0]
    for t in range(trials):
        s = rng.integers(0, 2, B).astype(bool)
        if not s.any():
            s[rng.integers(B)] = True
        q = np.bitwise_xor.reduce(R[s], axis=0)
        lhs = np.bitwise_xor.reduce(Out[s].reshape(int(s.sum()), -1).view(np.uint64), axis=0)
        rhs = oracle.read(T, n, d, z, q).view(np.uint64)
        if not np.array_equal(lhs, rhs):
            return f"Freivalds trial {t} differs"
    return None


def check_generated_table(task):
    """task = (tag, n, d, z, seed, table, R, outs, rows, trials, check_seed):
    regenerate table `table` of workload `seed` on the host and check every
    reply array in `outs` on the sampled rows and with `trials` GF(2)
    Freivalds trials.  Returns (tag, None) or (tag, message)."""
    from paper_2001_08250_gb300 import synth
    tag, n, d, z, seed, table, R, outs, rows, trials, check_seed = task
    T = synth.table_bytes(n, d, z, seed=seed, table=table)
    for k, Out in enumerate(outs):
        msg = _rows_and_freivalds(T, n, d, z, R, Out, rows, trials, check_seed + k)
        if msg:
            return tag, f"output {k}: {msg}"
    return tag, None


def check_mapped_table(task):
    """task = (tag, dir, n, d, z, rows, trials, check_seed): the same checks
    against the table, requests and replies the parent wrote to `dir`
    (table.bin raw bytes, R.npy, Out.npy), mapped read-only."""
    tag, path, n, d, z, rows, trials, check_seed = task
    T = np.memmap(os.path.join(path, "table.bin"), dtype=np.uint8, mode="r", shape=(n, d * z))
    R = np.load(os.path.join(path, "R.npy"), mmap_mode="r")
    Out = np.load(os.path.join(path, "Out.npy"), mmap_mode="r")
    return tag, _rows_and_freivalds(T, n, d, z, np.asarray(R), np.asarray(Out), rows, trials,
                                    check_seed)


def run_pool(fn, tasks, workers: int | None = None):
    """Results of fn over tasks in a spawn pool (in task order)."""
    workers = workers or max(1, min(8, (os.cpu_count() or 2) - 1))
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(fn, tasks, chunksize=1)
