"""Shared helpers of the GPU parity tests (test harness only)."""

import numpy as np

import oracle


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def to_dev(a: np.ndarray):
    torch = require_cuda()
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def dev_out(B: int, row_bytes: int):
    torch = require_cuda()
    return torch.empty((B, row_bytes), dtype=torch.uint8, device="cuda")


def to_host(t) -> np.ndarray:
    return t.cpu().numpy()


def freivalds(T, n, d, z, R, Out, trials, seed):
    """GF(2) Freivalds check of Out = R (x) T: for random subsets S of the
    requests, XOR_{b in S} Out[b] must equal the oracle's answer to
    XOR_{b in S} R[b] (the server answer is linear over XOR).  A wrong Out
    passes one trial with probability <= 1/2."""
    rng = np.random.default_rng(seed)
    B = R.shape[0]
    for _ in range(trials):
        s = rng.integers(0, 2, B).astype(bool)
        if not s.any():
            s[rng.integers(B)] = True
        q = np.bitwise_xor.reduce(R[s], axis=0)
        lhs = np.bitwise_xor.reduce(Out[s].reshape(int(s.sum()), -1).view(np.uint64), axis=0)
        rhs = oracle.read(T, n, d, z, q).view(np.uint64)
        assert np.array_equal(lhs, rhs)


def check_rows(T, n, d, z, R, Out, rows):
    for b in rows:
        exp = oracle.read(T, n, d, z, R[b])
        assert np.array_equal(Out[b], exp), f"row {b} differs"
