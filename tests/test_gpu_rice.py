"""GPU parity of the compressed GetUpdates encoding (Section 7's compressed
interest-vector deltas; the Golomb-Rice code of the gaps between set bits)
against the oracle, through the C ABI: the device stream must equal the
oracle's byte for byte (with the same bit count, set-bit count and
parameter) on random vectors of several sizes and densities, on the global
interest vector and every delta of a live window, and must decode back to
the vector."""

import ctypes

import numpy as np
import pytest

import oracle
from gpu_helpers import require_cuda
from paper_2001_08250_gb300 import synth, talekpir

pytestmark = pytest.mark.gpu


def _vec(m, density, seed):
    u = synth.uniform01(m, synth.stream_key(seed, 1, 77))
    v = np.zeros((m + 63) // 64, dtype=np.uint64)
    for p in np.nonzero(u < density)[0]:
        v[p // 64] |= np.uint64(1) << np.uint64(p % 64)
    return v


def _device_encode(v, m, k, cap):
    torch = require_cuda()
    dv = torch.from_numpy(v.view(np.int64)).cuda()
    out = torch.zeros(cap // 4, dtype=torch.int32, device="cuda")
    res = torch.zeros(3, dtype=torch.int64, device="cuda")
    talekpir.rice_encode_async(dv, m, out, cap, res, k)
    r = res.cpu().numpy().view(np.uint64)
    return out.cpu().numpy().view(np.uint8), int(r[0]), int(r[1]), int(r[2])


@pytest.mark.parametrize("m,density,seed", [(1, 1.0, 1), (63, 0.5, 2), (64, 1.0, 3),
                                             (1000, 0.02, 4), (4097, 0.3, 5), (65536, 0.001, 6),
                                             (1 << 20, 0.004, 7), (1 << 20, 0.5, 8),
                                             (3 << 20, 0.0002, 9), (777, 0.0, 10)])
@pytest.mark.parametrize("k", [-1, 0, 5, 20])
def test_rice_stream_bit_exact(m, density, seed, k):
    v = _vec(m, density, seed)
    exp, enb, ecnt, ek = oracle.rice_encode(v, m, None if k < 0 else k)
    cap = (len(exp) + 64) // 4 * 4 + 64
    got, nb, cnt, kk = _device_encode(v, m, k, cap)
    assert (nb, cnt, kk) == (enb, ecnt, ek)
    assert np.array_equal(got[:len(exp)], exp)
    assert not got[len(exp):].any()
    assert np.array_equal(oracle.rice_decode(got[:len(exp)], nb, kk, cnt, m), v)


def test_bits_past_m_ignored_and_overflow_reported():
    m = 100
    v = np.array([np.uint64(0xFFFFFFFFFFFFFFFF), np.uint64(0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
    exp, enb, ecnt, ek = oracle.rice_encode(v, m, 0)
    got, nb, cnt, kk = _device_encode(v, m, 0, 64)
    assert (nb, cnt) == (enb, ecnt) == (100, 100)
    assert np.array_equal(got[:len(exp)], exp)
    # a stream longer than the buffer: reported, nothing written past the end
    v2 = _vec(4096, 0.5, 11)
    got2, nb2, cnt2, _ = _device_encode(v2, 4096, 12, 64)
    assert nb2 == (1 << 64) - 1 and cnt2 > 0


def test_compressed_getupdates_global_vector_and_window_deltas():
    """Writes with k = 4 positions in m = 2^20 into a window of 4 deltas of 500
    writes: the compressed global vector and each delta equal the oracle's
    encoding of the oracle's vectors."""
    require_cuda()
    m, kpos, window, per, writes = 1 << 20, 4, 4, 500, 1700
    db = talekpir.DB(64, 4, 64)
    db.bloom_create(m, kpos, window, per)
    ob = oracle.Bloom(m, kpos, window, per)
    keys = synth.write_keys(writes, seed=12)
    pos = synth.bloom_positions(keys, m, kpos)
    for i in range(0, writes, 100):
        assert db.bloom_insert_batch(pos[i:i + 100]) == talekpir.OK
        for p in pos[i:i + 100]:
            ob.insert(p)
    vecs = [ob.get()] + [ob.delta(a) for a in range(1, window + 1)]
    for which, v in enumerate(vecs):
        stream, nb, cnt, k = db.bloom_get_compressed(which)
        exp, enb, ecnt, ek = oracle.rice_encode(v, m)
        assert (nb, cnt, k) == (enb, ecnt, ek), which
        assert np.array_equal(stream, exp), which
    # a too-small buffer is an error, not a truncated stream
    L = talekpir.lib()
    small = np.zeros(16, dtype=np.uint8)
    nb = ctypes.c_uint64()
    assert L.tpir_bloom_get_compressed(db.h, 0, -1, small.ctypes.data, 16, ctypes.byref(nb),
                                       None, None) == talekpir.ENOMEM
    assert L.tpir_bloom_get_compressed(db.h, window + 1, -1, small.ctypes.data, 16, None, None,
                                       None) == talekpir.EINVAL
    db.close()
    assert talekpir.device_status() == talekpir.OK
